"""Object wrappers over the C ABI (handles) and torch conveniences.

``Grid`` -> ``Mesh`` -> ``Fvm`` mirrors the paper's Grid -> Mesh ->
FunctionSpace workflow (Sec. 2.3, Fig. 2).  The operator methods of ``Fvm``
take torch CUDA tensors shaped [nnodes, ld] (field[node][level], levels
innermost) and call the C ABI on torch's current stream; torch only provides
the device memory and the stream.  ``GradientFn`` / ``DivergenceFn`` wrap the
forward kernels and their hand-written adjoint kernels as autograd functions;
``CurlFn`` and ``LaplacianFn`` take their backward passes from the same
adjoint kernels (curl(u, v) = D(v, -u), L = D G).  ``Remap`` interpolates
between grids.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi
from .capi import ATLAS_BF16, ATLAS_F32, ATLAS_F64

R_EARTH = 6371220.0

PROJECTIONS = {"rotated_lonlat": capi.ATLAS_PROJ_ROTATED_LONLAT, "mercator": capi.ATLAS_PROJ_MERCATOR,
               "lambert_conformal": capi.ATLAS_PROJ_LAMBERT_CONFORMAL,
               "polar_stereographic": capi.ATLAS_PROJ_POLAR_STEREOGRAPHIC}

OPS = {"gradient": capi.ATLAS_OP_GRADIENT, "divergence": capi.ATLAS_OP_DIVERGENCE,
       "gradient_adjoint": capi.ATLAS_OP_GRADIENT_ADJOINT,
       "divergence_adjoint": capi.ATLAS_OP_DIVERGENCE_ADJOINT, "laplacian": capi.ATLAS_OP_LAPLACIAN,
       "curl": capi.ATLAS_OP_CURL, "vector_gradient": capi.ATLAS_OP_VECTOR_GRADIENT,
       "curl_adjoint": capi.ATLAS_OP_CURL_ADJOINT}


def _view(ptr, ctype, n, shape=None, dtype=None):
    if n == 0:
        return np.zeros(shape or (0,), dtype=dtype)
    arr = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctype)), shape=(n,))
    arr = arr.copy()
    return arr.reshape(shape) if shape else arr


class Grid:
    """Octahedral reduced Gaussian grid O<N>, or with ``regular=True`` the
    regular (full) Gaussian grid F<N> (a point set for remapping targets);
    library-owned handle."""

    def __init__(self, N: int, regular: bool = False):
        h = ctypes.c_void_p()
        if regular:
            capi.atlas_grid_regular_gaussian(int(N), ctypes.byref(h))
        else:
            capi.atlas_grid_octahedral(int(N), ctypes.byref(h))
        self.handle = h
        self.N = int(N)
        self.regular = bool(regular)
        nn = ctypes.c_int64()
        nl = ctypes.c_int()
        capi.atlas_grid_info(h, ctypes.byref(nn), ctypes.byref(nl), None, None, None)
        self.nnodes, self.nlat = nn.value, nl.value
        self.projection = None

    @classmethod
    def regional(cls, projection: str, nx: int, ny: int, xmin: float, xmax: float, ymin: float, ymax: float, *,
                 radius: float = R_EARTH, lon0: float = 0.0, lat0: float = 45.0,
                 south_pole=(0.0, -90.0)) -> "Grid":
        """Regional (limited-area) grid: a rectangle of a projection's plane
        with nx points per row and ny rows.  ``projection`` is
        "rotated_lonlat" (x, y in rotated degrees; ``south_pole`` = the
        rotated south pole's (lon, lat) in degrees), "mercator" (x, y in
        metres on a sphere of ``radius``, central longitude ``lon0``),
        "lambert_conformal" (the same plus the tangent latitude ``lat0``) or
        "polar_stereographic" (the same, tangent at the pole ``lat0`` = 90
        or -90)."""
        code = PROJECTIONS[projection]
        if code == capi.ATLAS_PROJ_ROTATED_LONLAT:
            tail = (float(south_pole[0]), float(south_pole[1]), 0.0, 0.0)
        else:
            tail = (float(radius), float(lon0), float(lat0), 0.0)
        prm = (ctypes.c_double * 8)(float(xmin), float(xmax), float(ymin), float(ymax), *tail)
        h = ctypes.c_void_p()
        capi.atlas_grid_regional(code, int(nx), int(ny), ctypes.cast(prm, ctypes.c_void_p), ctypes.byref(h))
        self = cls.__new__(cls)
        self.handle = h
        self.N = 0
        self.regular = False
        self.projection = projection
        self.nx, self.ny = int(nx), int(ny)
        nn = ctypes.c_int64()
        nl = ctypes.c_int()
        capi.atlas_grid_info(h, ctypes.byref(nn), ctypes.byref(nl), None, None, None)
        self.nnodes, self.nlat = nn.value, nl.value
        return self

    def arrays(self):
        pl, ll, lat = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        capi.atlas_grid_info(self.handle, None, None, ctypes.byref(pl), ctypes.byref(ll), ctypes.byref(lat))
        lonlat = _view(ll, ctypes.c_double, 2 * self.nnodes, (self.nnodes, 2))
        out = dict(pl=_view(pl, ctypes.c_int32, self.nlat), lat=_view(lat, ctypes.c_double, self.nlat),
                   lon=lonlat[:, 0].copy(), lat_node=lonlat[:, 1].copy())
        if self.projection is not None:
            xy, sc = ctypes.c_void_p(), ctypes.c_void_p()
            capi.atlas_grid_regional_info(self.handle, None, None, None, ctypes.byref(xy), ctypes.byref(sc))
            out["xy"] = _view(xy, ctypes.c_double, 2 * self.nnodes, (self.nnodes, 2))
            out["scale"] = _view(sc, ctypes.c_double, 2 * self.nnodes, (self.nnodes, 2))
        return out

    def close(self):
        if self.handle is not None and self.handle.value:
            capi.atlas_grid_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """Zipper triangulation + pole edges + CSR of a Grid."""

    def __init__(self, grid: Grid):
        h = ctypes.c_void_p()
        capi.atlas_mesh_build(grid.handle, ctypes.byref(h))
        self.handle = h
        self.grid = grid
        ne, nt = ctypes.c_int64(), ctypes.c_int64()
        capi.atlas_mesh_info(h, ctypes.byref(ne), ctypes.byref(nt), None, None, None, None, None, None)
        self.nedges, self.ntri = ne.value, nt.value

    def arrays(self):
        ptrs = [ctypes.c_void_p() for _ in range(6)]
        capi.atlas_mesh_info(self.handle, None, None, *(ctypes.byref(p) for p in ptrs))
        V, E, T = self.grid.nnodes, self.nedges, self.ntri
        e2n, pole, ptr, n2e, sgn, tri = ptrs
        return dict(e2n=_view(e2n, ctypes.c_int32, 2 * E, (E, 2)), is_pole=_view(pole, ctypes.c_uint8, E),
                    n2e_ptr=_view(ptr, ctypes.c_int32, V + 1), n2e=_view(n2e, ctypes.c_int32, 2 * E),
                    n2e_sign=_view(sgn, ctypes.c_int8, 2 * E), tri=_view(tri, ctypes.c_int32, 3 * T, (T, 3)))

    def close(self):
        if self.handle is not None and self.handle.value:
            capi.atlas_mesh_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _torch():
    import torch
    return torch


_DTYPES = None


def _dtype_code(t):
    global _DTYPES
    torch = _torch()
    if _DTYPES is None:
        _DTYPES = {torch.float32: ATLAS_F32, torch.float64: ATLAS_F64, torch.bfloat16: ATLAS_BF16}
    try:
        return _DTYPES[t.dtype]
    except KeyError:
        raise TypeError("fields must be float32, float64 or bfloat16 (got %s)" % t.dtype) from None


def _stream():
    return _torch().cuda.current_stream().cuda_stream


class Fvm:
    """Median-dual geometry of a Mesh with radius R, plus the operator calls."""

    def __init__(self, mesh: Mesh, radius: float = R_EARTH):
        h = ctypes.c_void_p()
        capi.atlas_fvm_build_dual(mesh.handle, float(radius), ctypes.byref(h))
        self.handle = h
        self.mesh = mesh
        self.grid = mesh.grid
        self.R = float(radius)
        self.nnodes = mesh.grid.nnodes

    # ----------------------------------------------------------- geometry
    def arrays(self):
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        capi.atlas_fvm_info(self.handle, *(ctypes.byref(p) for p in ptrs))
        V, E = self.nnodes, self.mesh.nedges
        out = dict(V=_view(ptrs[0], ctypes.c_double, V), S=_view(ptrs[1], ctypes.c_double, 2 * E, (E, 2)),
                   coslat=_view(ptrs[2], ctypes.c_double, V), pole_nphi=_view(ptrs[3], ctypes.c_double, V))
        if self.grid.projection is not None:
            a, sb = ctypes.c_void_p(), ctypes.c_void_p()
            capi.atlas_fvm_regional_info(self.handle, ctypes.byref(a), ctypes.byref(sb))
            out["area"] = _view(a, ctypes.c_double, V)
            out["Sb"] = _view(sb, ctypes.c_double, 2 * E, (E, 2))
        return out

    def save(self, path):
        """Write the host grid, mesh and dual to ``path`` (``load_fvm`` reads it)."""
        capi.atlas_fvm_save(self.handle, str(path).encode())

    def check(self):
        """Consistency check of the host geometry (CSR and closure of every
        dual cell); returns the largest relative closure residual, raises
        AtlasError naming the first bad node."""
        worst = ctypes.c_double()
        capi.atlas_fvm_check(self.handle, ctypes.byref(worst))
        return worst.value

    def prepare(self, ops=("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint"),
                dtypes=(ATLAS_F32,)):
        om = 0
        for o in ops:
            om |= 1 << OPS[o]
        dm = 0
        for d in dtypes:
            dm |= 1 << d
        capi.atlas_fvm_prepare(self.handle, om, dm)

    def stencil_table(self, op):
        """FP64 host table of one operator's node stencil (inspection)."""
        code = OPS.get(op, op)
        nnz, nin, nout = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        capi.atlas_fvm_stencil_table(self.handle, code, ctypes.byref(nnz), ctypes.byref(nin), ctypes.byref(nout),
                                     None, None, None, None)
        V, n = self.nnodes, nnz.value
        ptr = np.empty(V + 1, np.int32)
        nbr = np.empty(max(n, 1), np.int32)
        w = np.empty((max(n, 1), 2))
        b = np.empty((V, 2))
        capi.atlas_fvm_stencil_table(self.handle, code, None, None, None, ptr.ctypes.data, nbr.ctypes.data,
                                     w.ctypes.data, b.ctypes.data)
        return dict(ptr=ptr, nbr=nbr[:n], w=w[:n], b=b, nin=nin.value, nout=nout.value)

    def tile_table(self, op, groups_per_tile=7, unions=True, rows_per_tile=1):
        """The FP32 tile table of op's node-group kernels (host only): head
        [ntiles][72], blob (uint32 words), and the units (runs of grid rows
        whose tiles are consecutive): unit_first [nunits + 1] (first node,
        then nnodes), unit_tile [nunits + 1] (first tile, then ntiles); see
        atlas_fvm_tile_table."""
        code = OPS.get(op, op)
        nt, nw, nu = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        args = (self.handle, code, int(groups_per_tile), int(rows_per_tile), int(bool(unions)))
        capi.atlas_fvm_tile_table(*args, ctypes.byref(nt), ctypes.byref(nw), None, None, ctypes.byref(nu), None, None)
        head = np.empty((max(nt.value, 1), 72), np.int32)
        blob = np.empty(max(nw.value, 1), np.uint32)
        uf = np.empty(nu.value + 1, np.int64)
        ut = np.empty(nu.value + 1, np.int32)
        capi.atlas_fvm_tile_table(*args, None, None, head.ctypes.data, blob.ctypes.data, None, uf.ctypes.data,
                                  ut.ctypes.data)
        return dict(head=head[:nt.value], blob=blob[:nw.value], unit_first=uf, unit_tile=ut)

    def tile_union_groups(self, op, dtype=ATLAS_F32):
        """How many groups of op's node-group tables are stored in union
        form (each distinct neighbour row read once for the group's four
        nodes); 0 when there are none."""
        n = ctypes.c_int64()
        capi.atlas_fvm_tile_union_groups(self.handle, OPS.get(op, op), int(dtype), ctypes.byref(n))
        return n.value

    def tile_info(self, op, nlev, ld, dtype=ATLAS_F32):
        """Launch shape of the node-group kernel of op on [nnodes, ld] fields
        of nlev levels: blocks per SM, stages, shared memory per block,
        the most rows a tile stages (all 0 when it runs per node)."""
        b, s = ctypes.c_int(), ctypes.c_int()
        m, r = ctypes.c_int64(), ctypes.c_int64()
        capi.atlas_fvm_tile_info(self.handle, OPS.get(op, op), int(dtype), int(nlev), int(ld), ctypes.byref(b),
                                 ctypes.byref(s), ctypes.byref(m), ctypes.byref(r))
        return dict(blocks_per_sm=b.value, stages=s.value, smem=m.value, max_rows=r.value)

    def group_table(self, op):
        """The FP64 node-group table of one operator (host only): head
        [ngroups][4], hdr [nent], w [nent][4][2] (see atlas_fvm_group_table)."""
        code = OPS.get(op, op)
        ng, ne = ctypes.c_int64(), ctypes.c_int64()
        capi.atlas_fvm_group_table(self.handle, code, ctypes.byref(ng), ctypes.byref(ne), None, None, None)
        head = np.empty((max(ng.value, 1), 4), np.int32)
        hdr = np.empty(max(ne.value, 1), np.uint32)
        w = np.empty((max(ne.value, 1), 4, 2))
        capi.atlas_fvm_group_table(self.handle, code, None, None, head.ctypes.data, hdr.ctypes.data, w.ctypes.data)
        return dict(head=head[:ng.value], hdr=hdr[:ne.value], w=w[:ne.value])

    def set_launch(self, op, vec=0, batch=0, threads=0, blocks_per_sm=0, tile_passes=0, dtype=-1):
        """Launch shape of one operator for one storage dtype (ATLAS_F32 /
        ATLAS_F64 / ATLAS_BF16) or, with dtype=-1, for all of them."""
        capi.atlas_fvm_set_launch(self.handle, OPS.get(op, op), int(dtype), int(vec), int(batch), int(threads),
                                  int(blocks_per_sm), int(tile_passes))

    def set_group(self, op, enable=-1, blocks_per_sm=0, groups_per_tile=0, dtype=-1, nodes_per_warp=0,
                  rows_per_tile=0):
        """Use the shared-memory node-group kernels for one operator by
        default (enable 1: one-ring operators on fields of more than 80
        levels for FP32 and 96 for BF16, the Laplacian on any), on every
        field they apply to (2), or
        the per-node kernels only (0; -1 keeps),
        with at most
        blocks_per_sm blocks per SM (1 or 2; 0 keeps), groups_per_tile
        groups of four nodes per tile (1..11; 0 keeps), nodes_per_warp
        nodes per consumer warp (4 or 2; 0 keeps) and tiles spanning
        rows_per_tile grid rows (1..3, groups_per_tile split between them;
        0 keeps), for one storage dtype or, with dtype=-1, all of them."""
        capi.atlas_fvm_set_group(self.handle, OPS.get(op, op), int(dtype), int(enable), int(blocks_per_sm),
                                 int(groups_per_tile), int(nodes_per_warp), int(rows_per_tile))

    def group_table(self, op):
        """The FP64 node-group table of one operator (host only): head
        [ngroups][4], hdr [nent], w [nent][4][2] (see atlas_fvm_group_table)."""
        code = OPS.get(op, op)
        ng, ne = ctypes.c_int64(), ctypes.c_int64()
        capi.atlas_fvm_group_table(self.handle, code, ctypes.byref(ng), ctypes.byref(ne), None, None, None)
        head = np.empty((max(ng.value, 1), 4), np.int32)
        hdr = np.empty(max(ne.value, 1), np.uint32)
        w = np.empty((max(ne.value, 1), 4, 2))
        capi.atlas_fvm_group_table(self.handle, code, None, None, head.ctypes.data, hdr.ctypes.data, w.ctypes.data)
        return dict(head=head[:ng.value], hdr=hdr[:ne.value], w=w[:ne.value])

    def set_launch(self, op, vec=0, batch=0, threads=0, blocks_per_sm=0, tile_passes=0, dtype=-1):
        """Launch shape of one operator for one storage dtype (ATLAS_F32 /
        ATLAS_F64 / ATLAS_BF16) or, with dtype=-1, for all of them."""
        capi.atlas_fvm_set_launch(self.handle, OPS.get(op, op), int(dtype), int(vec), int(batch), int(threads),
                                  int(blocks_per_sm), int(tile_passes))

    # ---------------------------------------------------------- operators
    def _check(self, *ts):
        t0 = ts[0]
        for t in ts:
            if not t.is_cuda or t.dim() != 2 or t.shape[0] != self.nnodes or t.stride(1) != 1:
                raise ValueError("fields must be CUDA tensors [nnodes=%d, ld] with unit level stride" % self.nnodes)
            if t.dtype != t0.dtype or t.stride(0) != t0.stride(0):
                raise ValueError("all fields of one call need the same dtype and leading dimension")
        return _dtype_code(t0), t0.stride(0)

    def _out(self, like, out):
        return _torch().empty_like(like) if out is None else out

    def gradient(self, f, nlev=None, out=None):
        gx, gy = out if out is not None else (self._out(f, None), self._out(f, None))
        dt, ld = self._check(f, gx, gy)
        capi.atlas_nabla_gradient(self.handle, f.data_ptr(), gx.data_ptr(), gy.data_ptr(),
                                  f.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return gx, gy

    def divergence(self, u, v, nlev=None, out=None):
        d = self._out(u, out)
        dt, ld = self._check(u, v, d)
        capi.atlas_nabla_divergence(self.handle, u.data_ptr(), v.data_ptr(), d.data_ptr(),
                                    u.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return d

    def laplacian(self, f, nlev=None, out=None):
        lap = self._out(f, out)
        dt, ld = self._check(f, lap)
        capi.atlas_nabla_laplacian(self.handle, f.data_ptr(), lap.data_ptr(),
                                   f.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return lap

    def gradient_adjoint(self, gx, gy, nlev=None, out=None):
        f = self._out(gx, out)
        dt, ld = self._check(gx, gy, f)
        capi.atlas_nabla_gradient_adjoint(self.handle, gx.data_ptr(), gy.data_ptr(), f.data_ptr(),
                                          gx.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return f

    def divergence_adjoint(self, d, nlev=None, out=None):
        u, v = out if out is not None else (self._out(d, None), self._out(d, None))
        dt, ld = self._check(d, u, v)
        capi.atlas_nabla_divergence_adjoint(self.handle, d.data_ptr(), u.data_ptr(), v.data_ptr(),
                                            d.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return u, v

    def curl(self, u, v, nlev=None, out=None):
        z = self._out(u, out)
        dt, ld = self._check(u, v, z)
        capi.atlas_nabla_curl(self.handle, u.data_ptr(), v.data_ptr(), z.data_ptr(),
                              u.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return z

    def curl_adjoint(self, z, nlev=None, out=None):
        u, v = out if out is not None else (self._out(z, None), self._out(z, None))
        dt, ld = self._check(z, u, v)
        capi.atlas_nabla_curl_adjoint(self.handle, z.data_ptr(), u.data_ptr(), v.data_ptr(),
                                      z.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return u, v

    def integral(self, x, nlev=None, node0=0, count=None, out=None, ws=None):
        """FP64 volume-weighted sums over nodes node0 .. node0+count-1 of the
        rows of x (x's first row is node node0's): a float64 CUDA tensor
        [nlev], out[k] = sum_i V_i x[i, k]."""
        torch = _torch()
        if not x.is_cuda or x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("x must be a CUDA tensor [rows, ld] with unit level stride")
        count = x.shape[0] if count is None else int(count)
        nlev = x.shape[1] if nlev is None else int(nlev)
        if count > x.shape[0]:
            raise ValueError("count exceeds the rows of x")
        out = torch.empty(nlev, dtype=torch.float64, device=x.device) if out is None else out
        need = capi.atlas_fvm_integral_workspace_bytes(self.handle, nlev)
        if ws is None:
            ws = torch.empty(max(need // 8, 1), dtype=torch.float64, device=x.device)
        capi.atlas_fvm_integral(self.handle, x.data_ptr(), int(node0), count, nlev, x.stride(0), _dtype_code(x),
                                out.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(), _stream())
        return out

    def vector_gradient(self, u, v, nlev=None, out=None):
        """(ux, uy, vx, vy): gradients of both components of a tangent vector."""
        outs = out if out is not None else tuple(self._out(u, None) for _ in range(4))
        dt, ld = self._check(u, v, *outs)
        capi.atlas_nabla_vector_gradient(self.handle, u.data_ptr(), v.data_ptr(), *(o.data_ptr() for o in outs),
                                         u.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return tuple(outs)

    # edge-based two-kernel forms
    def workspace(self, op, ld, dtype_code):
        torch = _torch()
        n = capi.atlas_nabla_workspace_bytes(self.handle, OPS.get(op, op), 0, int(ld), int(dtype_code))
        return torch.empty(max(int(n), 256), dtype=torch.uint8, device="cuda")

    def gradient_edges(self, f, nlev=None, ws=None, out=None, averaged=False):
        """Edge-flux + node-gather gradient; averaged=True takes the edge flux
        in the averaged form S_e (f_a + f_b)/2 instead of the difference form."""
        gx, gy = out if out is not None else (self._out(f, None), self._out(f, None))
        dt, ld = self._check(f, gx, gy)
        ws = self.workspace("gradient", ld, dt) if ws is None else ws
        call = capi.atlas_nabla_gradient_edges_averaged if averaged else capi.atlas_nabla_gradient_edges
        call(self.handle, f.data_ptr(), gx.data_ptr(), gy.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(),
             f.shape[1] if nlev is None else nlev, ld, dt, _stream())
        return gx, gy

    def divergence_edges(self, u, v, nlev=None, ws=None, out=None):
        d = self._out(u, out)
        dt, ld = self._check(u, v, d)
        ws = self.workspace("divergence", ld, dt) if ws is None else ws
        capi.atlas_nabla_divergence_edges(self.handle, u.data_ptr(), v.data_ptr(), d.data_ptr(), ws.data_ptr(),
                                          ws.numel() * ws.element_size(), u.shape[1] if nlev is None else nlev,
                                          ld, dt, _stream())
        return d

    def laplacian_edges(self, f, nlev=None, ws=None, out=None):
        lap = self._out(f, out)
        dt, ld = self._check(f, lap)
        ws = self.workspace("laplacian", ld, dt) if ws is None else ws
        capi.atlas_nabla_laplacian_edges(self.handle, f.data_ptr(), lap.data_ptr(), ws.data_ptr(),
                                         ws.numel() * ws.element_size(), f.shape[1] if nlev is None else nlev,
                                         ld, dt, _stream())
        return lap

    def close(self):
        if self.handle is not None and self.handle.value:
            capi.atlas_fvm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Remap:
    """Linear interpolation, in three-dimensional space over the sphere, from
    the nodes of ``mesh`` to the points of ``grid`` (located and weighted on
    the host, applied by a CUDA kernel)."""

    def __init__(self, mesh: Mesh, grid: Grid):
        h = ctypes.c_void_p()
        capi.atlas_remap_create(mesh.handle, grid.handle, ctypes.byref(h))
        self.handle, self.mesh, self.grid = h, mesh, grid
        n = ctypes.c_int64()
        capi.atlas_remap_info(h, ctypes.byref(n), None, None)
        self.ntgt = n.value

    def tables(self):
        """(nodes [T][3] int32, weights [T][3] float64), copies."""
        pn, pw = ctypes.c_void_p(), ctypes.c_void_p()
        capi.atlas_remap_info(self.handle, None, ctypes.byref(pn), ctypes.byref(pw))
        return (_view(pn, ctypes.c_int32, 3 * self.ntgt, (self.ntgt, 3)),
                _view(pw, ctypes.c_double, 3 * self.ntgt, (self.ntgt, 3)))

    def apply(self, src, nlev=None, out=None, ld_dst=None):
        """src: CUDA tensor [source nodes, ld]; returns [targets, ld_dst]."""
        torch = _torch()
        if not src.is_cuda or src.dim() != 2 or src.stride(1) != 1:
            raise ValueError("src must be a CUDA tensor [nodes, ld] with unit level stride")
        nlev = src.shape[1] if nlev is None else int(nlev)
        if out is None:
            out = torch.empty((self.ntgt, src.stride(0) if ld_dst is None else int(ld_dst)), dtype=src.dtype,
                              device=src.device)
        if out.dtype != src.dtype or out.shape[0] != self.ntgt or out.stride(1) != 1:
            raise ValueError("out must be [%d targets, ld] of the source dtype" % self.ntgt)
        capi.atlas_remap_apply(self.handle, src.data_ptr(), out.data_ptr(), nlev, src.stride(0), out.stride(0),
                               _dtype_code(src), _stream())
        return out

    def close(self):
        if self.handle is not None and self.handle.value:
            capi.atlas_remap_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_fvm(N: int, radius: float = R_EARTH, regular: bool = False) -> Fvm:
    """Grid O<N> (or F<N> with regular=True) -> Mesh -> median-dual Fvm in one call."""
    g = Grid(N, regular=regular)
    m = Mesh(g)
    return Fvm(m, radius)


def load_fvm(path) -> Fvm:
    """An Fvm (with its Grid and Mesh) read from a file written by ``Fvm.save``."""
    hg, hm, hf = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    capi.atlas_fvm_load(str(path).encode(), ctypes.byref(hg), ctypes.byref(hm), ctypes.byref(hf))
    g = Grid.__new__(Grid)
    g.handle = hg
    nn, nl = ctypes.c_int64(), ctypes.c_int()
    capi.atlas_grid_info(hg, ctypes.byref(nn), ctypes.byref(nl), None, None, None)
    g.nnodes, g.nlat = nn.value, nl.value
    proj, nx, ny = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    try:
        capi.atlas_grid_regional_info(hg, ctypes.byref(proj), ctypes.byref(nx), ctypes.byref(ny), None, None)
        g.projection = {v: k for k, v in PROJECTIONS.items()}[proj.value]
        g.nx, g.ny, g.N, g.regular = nx.value, ny.value, 0, False
    except capi.AtlasError:  # a global grid: O<N> or F<N>
        g.projection = None
        g.N = g.nlat // 2
        g.regular = g.nnodes == 8 * g.N * g.N
    m = Mesh.__new__(Mesh)
    m.handle, m.grid = hm, g
    ne, nt = ctypes.c_int64(), ctypes.c_int64()
    capi.atlas_mesh_info(hm, ctypes.byref(ne), ctypes.byref(nt), None, None, None, None, None, None)
    m.nedges, m.ntri = ne.value, nt.value
    f = Fvm.__new__(Fvm)
    f.handle, f.mesh, f.grid, f.nnodes = hf, m, g, g.nnodes
    r = ctypes.c_double()
    capi.atlas_fvm_radius(hf, ctypes.byref(r))
    f.R = r.value
    return f


def build_fvm_regional(projection: str, nx: int, ny: int, xmin: float, xmax: float, ymin: float, ymax: float,
                       radius: float = R_EARTH, **proj) -> Fvm:
    """Regional Grid (see ``Grid.regional``) -> Mesh -> Fvm in one call; the
    dual's radius is the projection's."""
    g = Grid.regional(projection, nx, ny, xmin, xmax, ymin, ymax, radius=radius, **proj)
    return Fvm(Mesh(g), radius)


def measure_fp64_rate(iters=1 << 14, blocks_per_sm=8, reps=3):
    """Measured FP64 FMA rate of the current device (TFLOP/s): the library's
    FP64 FMA kernel on every SM, timed with CUDA events after a warm-up."""
    torch = _torch()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, threads = sms * blocks_per_sm, 256
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    s = _stream()
    run = lambda: capi.atlas_fp64_fma_rate_kernel(out.data_ptr(), blocks, threads, int(iters), s)
    run()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        run()
    b.record()
    b.synchronize()
    sec = a.elapsed_time(b) * 1e-3 / reps
    return 16.0 * iters * blocks * threads / sec / 1e12


def kernel_status(clear=True):
    """The device error word of the node-group kernels (0: no kernel gave up
    a wait); waits for the device.  clear resets it."""
    code = ctypes.c_uint(0)
    capi.atlas_kernel_status(ctypes.byref(code), 1 if clear else 0)
    return code.value


def field_sync(dst, src, nbytes, direction, stream=None):
    """One cudaMemcpyAsync (0 = H2D, 1 = D2H, 2 = D2D) on torch's current stream."""
    capi.atlas_field_sync(dst, src, int(nbytes), int(direction), _stream() if stream is None else stream)


# ---------------------------------------------------------------- autograd
def _make_autograd():
    torch = _torch()

    class GradientFn(torch.autograd.Function):
        """(gx, gy) = G f; backward f_bar = G^T (gx_bar, gy_bar) by the adjoint kernel."""

        @staticmethod
        def forward(ctx, f, fvm):
            ctx.fvm = fvm
            f = f.contiguous()
            out = (torch.zeros_like(f), torch.zeros_like(f))  # padding levels stay 0
            return fvm.gradient(f, out=out)

        @staticmethod
        def backward(ctx, gx_bar, gy_bar):
            fvm = ctx.fvm
            gx_bar = torch.zeros_like(gy_bar) if gx_bar is None else gx_bar.contiguous()
            gy_bar = torch.zeros_like(gx_bar) if gy_bar is None else gy_bar.contiguous()
            return fvm.gradient_adjoint(gx_bar, gy_bar, out=torch.zeros_like(gx_bar)), None

    class DivergenceFn(torch.autograd.Function):
        """d = D (u, v); backward (u_bar, v_bar) = D^T d_bar by the adjoint kernel."""

        @staticmethod
        def forward(ctx, u, v, fvm):
            ctx.fvm = fvm
            u = u.contiguous()
            return fvm.divergence(u, v.contiguous(), out=torch.zeros_like(u))

        @staticmethod
        def backward(ctx, d_bar):
            d_bar = d_bar.contiguous()
            out = (torch.zeros_like(d_bar), torch.zeros_like(d_bar))
            u_bar, v_bar = ctx.fvm.divergence_adjoint(d_bar, out=out)
            return u_bar, v_bar, None

    class CurlFn(torch.autograd.Function):
        """z = curl (u, v); backward (u_bar, v_bar) = C^T z_bar by the curl
        adjoint kernel."""

        @staticmethod
        def forward(ctx, u, v, fvm):
            ctx.fvm = fvm
            u = u.contiguous()
            return fvm.curl(u, v.contiguous(), out=torch.zeros_like(u))

        @staticmethod
        def backward(ctx, z_bar):
            z_bar = z_bar.contiguous()
            u_bar, v_bar = ctx.fvm.curl_adjoint(z_bar, out=(torch.zeros_like(z_bar), torch.zeros_like(z_bar)))
            return u_bar, v_bar, None

    class LaplacianFn(torch.autograd.Function):
        """l = L f with the fused two-ring table L = D G; backward
        f_bar = G^T (D^T l_bar) by the two adjoint kernels."""

        @staticmethod
        def forward(ctx, f, fvm):
            ctx.fvm = fvm
            f = f.contiguous()
            return fvm.laplacian(f, out=torch.zeros_like(f))

        @staticmethod
        def backward(ctx, l_bar):
            l_bar = l_bar.contiguous()
            u, v = ctx.fvm.divergence_adjoint(l_bar, out=(torch.zeros_like(l_bar), torch.zeros_like(l_bar)))
            return ctx.fvm.gradient_adjoint(u, v, out=torch.zeros_like(l_bar)), None

    return GradientFn, DivergenceFn, CurlFn, LaplacianFn


_AUTOGRAD = None


def gradient_fn(f, fvm: Fvm):
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD[0].apply(f, fvm)


def divergence_fn(u, v, fvm: Fvm):
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD[1].apply(u, v, fvm)


def curl_fn(u, v, fvm: Fvm):
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD[2].apply(u, v, fvm)


def laplacian_fn(f, fvm: Fvm):
    global _AUTOGRAD
    if _AUTOGRAD is None:
        _AUTOGRAD = _make_autograd()
    return _AUTOGRAD[3].apply(f, fvm)
