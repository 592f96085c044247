"""Measured error of every operator against the FP64 oracle.

The operators run in FP32 (and BF16 storage with FP32 arithmetic, and FP64)
while the method's geometry is FP64; each operator's error against the FP64
oracle is measured here on the benchmark's fields and reported:

* O320 x 137 levels, the full field: FP32, BF16-storage and FP64 paths, the
  oracle fed the same rounded inputs (upcast exactly);
* FP32 against the FP64 GPU path on the same FP32 inputs, O320 x 137;
* O1280 x 137 on sampled nodes (every polar-row node and the ends of every
  row included): FP32 and FP64;
* the edge-flux gradient in the averaged form S_e (f_a + f_b)/2 beside the
  difference form S_e (f_b - f_a)/2, FP32, O320 (sampled nodes): in FP32
  the averaged form's node sums cancel terms about R/h times larger than
  the result, which the difference form avoids.

Error = max |gpu - oracle| / max |oracle| per output component over all
nodes and levels.  The bars asserted are the parity tolerances (FP64 1e-13,
FP32 1e-5, BF16 2e-2); the averaged form's FP32 error is bounded only by
the cancellation estimate (below 2e-3).  With PRECISION_REPORT set to a file
name the table is also written there as JSON.  The oracle runs in a pool of
spawned worker processes over node chunks.
"""
import json
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

NLEV = 137
OPS = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint", "curl", "vector_gradient",
       "curl_adjoint")
COMPONENTS = {"gradient": ("gx", "gy"), "divergence": ("div",), "laplacian": ("lap",),
              "gradient_adjoint": ("f",), "divergence_adjoint": ("u", "v"), "curl": ("zeta",),
              "vector_gradient": ("ux", "uy", "vx", "vy"), "curl_adjoint": ("u", "v")}
REPORT = {}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _relmax(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def _bf16(x):
    """float32 -> nearest bfloat16 (ties to even), as float32: what the GPU
    stores for a float32 value."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _fields(N, kind, g=None):
    """The benchmark recipe's (f, u, v) on O<N> x 137 as the GPU path of
    `kind` reads them (fp32, bf16 rounded from fp32, or fp64); g: the
    oracle's grid arrays of O<N> (built when None)."""
    if g is None:
        from oracle.oracle import Mesh
        g = Mesh(N).grid()
    dt = np.float64 if kind == "fp64" else np.float32
    f = synthetic.level_scalar(g["lon"], g["lat_node"], NLEV, dt)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], NLEV, dt)
    if kind == "bf16":
        f, u, v = _bf16(f), _bf16(u), _bf16(v)
    return f, u, v


def _oracle_ops(om, f, u, v, nodes):
    return {"gradient": om.gradient(f, NLEV, nodes=nodes), "divergence": (om.divergence(u, v, NLEV, nodes=nodes),),
            "laplacian": (om.laplacian(f, NLEV, nodes=nodes),),
            "gradient_adjoint": (om.gradient_adjoint(u, v, NLEV, nodes=nodes),),
            "divergence_adjoint": om.divergence_adjoint(f, NLEV, nodes=nodes),
            "curl": (om.curl(u, v, NLEV, nodes=nodes),),
            "vector_gradient": om.vector_gradient(u, v, NLEV, nodes=nodes),
            "curl_adjoint": om.curl_adjoint(f, NLEV, nodes=nodes)}


def _oracle_chunk(args):
    """Worker: the oracle's outputs of every operator on nodes [n0, n1),
    the fields rebuilt from their seeds (nothing large crosses the pipe
    but the results)."""
    N, kind, n0, n1 = args
    from oracle.oracle import Mesh
    om = Mesh(N)
    f, u, v = _fields(N, kind, om.grid())
    out = _oracle_ops(om, f, u, v, np.arange(n0, n1, dtype=np.int64))
    return {op: tuple(np.asarray(x, np.float32 if kind != "fp64" else np.float64) for x in vals)
            for op, vals in out.items()}


def _oracle_all(N, kind, V):
    """Oracle outputs on every node, computed in spawned workers over node
    chunks (float32 results for the float32 and bfloat16 inputs: their
    error against the oracle is far above float32 rounding)."""
    workers = max(1, min(16, os.cpu_count() or 4))
    edges = np.linspace(0, V, workers + 1).astype(np.int64)
    chunks = [(N, kind, int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_oracle_chunk, chunks))
    return {op: tuple(np.concatenate([p[op][c] for p in parts]) for c in range(len(COMPONENTS[op]))) for op in OPS}


def _gpu_all(torch, fvm, tf, tu, tv):
    out = {"gradient": fvm.gradient(tf, NLEV), "divergence": (fvm.divergence(tu, tv, NLEV),),
           "laplacian": (fvm.laplacian(tf, NLEV),), "gradient_adjoint": (fvm.gradient_adjoint(tu, tv, NLEV),),
           "divergence_adjoint": fvm.divergence_adjoint(tf, NLEV), "curl": (fvm.curl(tu, tv, NLEV),),
           "vector_gradient": fvm.vector_gradient(tu, tv, NLEV), "curl_adjoint": fvm.curl_adjoint(tf, NLEV)}
    torch.cuda.synchronize()
    return out


def _dev(torch, x, ld, dt):
    """[V][nlev] -> CUDA [V][ld] of dtype dt; float32 data goes through
    float32 (so bfloat16 is rounded once, from float32)."""
    x = np.asarray(x)
    t = torch.from_numpy(np.ascontiguousarray(synthetic.padded(x, ld)))
    return t.to(dt).cuda()


def _errors(got, want, nodes_idx=None):
    res = {}
    for op in OPS:
        for c, name in enumerate(COMPONENTS[op]):
            g = got[op][c]
            if nodes_idx is not None:
                g = g.index_select(0, nodes_idx)
            res["%s.%s" % (op, name)] = _relmax(g[:, :NLEV].double().cpu().numpy(), want[op][c])
    return res


def _write_report():
    path = os.environ.get("PRECISION_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(REPORT, fh, indent=1, sort_keys=True)


def test_o320_full_field_fp32_bf16_fp64(torch, pfvm, omesh):
    fvm, g = pfvm(320), omesh(320).grid()
    base = {}
    for name, t_dt, ld, tol in (("fp32", torch.float32, 140, 1e-5), ("bf16", torch.bfloat16, 144, 2e-2),
                                ("fp64", torch.float64, 138, 1e-13)):
        f, u, v = _fields(320, name, g)
        tf, tu, tv = (_dev(torch, x, ld, t_dt) for x in (f, u, v))
        # the GPU holds exactly the values the oracle workers rebuild
        for a, b in ((tf, f), (tu, u), (tv, v)):
            assert np.array_equal(a[:, :NLEV].double().cpu().numpy(), np.asarray(b, np.float64))
        got = _gpu_all(torch, fvm, tf, tu, tv)
        want = _oracle_all(320, name, fvm.nnodes)
        err = _errors(got, want)
        REPORT["O320x137 full field %s vs oracle" % name] = err
        if name == "fp32":
            base = dict(f=f, u=u, v=v, got=got)
        del tf, tu, tv, got
        torch.cuda.empty_cache()
        assert max(err.values()) <= tol, (name, err)
    # FP32 against the FP64 GPU path on the same FP32 inputs
    tf, tu, tv = (_dev(torch, x, 138, torch.float64) for x in (base["f"], base["u"], base["v"]))
    ref = _gpu_all(torch, fvm, tf, tu, tv)
    err = {}
    for op in OPS:
        for c, name in enumerate(COMPONENTS[op]):
            err["%s.%s" % (op, name)] = _relmax(base["got"][op][c][:, :NLEV].double().cpu().numpy(),
                                                ref[op][c][:, :NLEV].cpu().numpy())
    REPORT["O320x137 full field fp32 vs fp64 GPU"] = err
    _write_report()
    assert max(err.values()) <= 1e-5, err


def test_o1280_sampled_fp32_fp64(torch, pfvm, omesh):
    fvm, om = pfvm(1280), omesh(1280)
    g = om.grid()
    off = np.concatenate([[0], np.cumsum(g["pl"])])
    nodes = synthetic.sample_nodes(om.nnodes, off, 3000)
    idx = torch.from_numpy(nodes).cuda()
    for name, t_dt, ld, tol in (("fp32", torch.float32, 140, 1e-5), ("fp64", torch.float64, 138, 1e-13)):
        f, u, v = _fields(1280, name, g)
        tf, tu, tv = (_dev(torch, x, ld, t_dt) for x in (f, u, v))
        got = _gpu_all(torch, fvm, tf, tu, tv)
        want = _oracle_ops(om, f, u, v, nodes)
        err = _errors(got, want, idx)
        REPORT["O1280x137 sampled (%d nodes) %s vs oracle" % (nodes.size, name)] = err
        del tf, tu, tv, got
        torch.cuda.empty_cache()
        _write_report()
        assert max(err.values()) <= tol, (name, err)


@pytest.mark.parametrize("N", [320])
def test_averaged_flux_gradient_fp32_error(torch, pfvm, omesh, N):
    """The averaged-form edge-flux gradient against the oracle's averaged
    Green-Gauss sum and the difference form against the oracle's
    closure-exact sum, both FP32 on the same inputs (sampled nodes)."""
    fvm, om = pfvm(N), omesh(N)
    g = om.grid()
    off = np.concatenate([[0], np.cumsum(g["pl"])])
    nodes = synthetic.sample_nodes(om.nnodes, off, 3000)
    idx = torch.from_numpy(nodes).cuda()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], NLEV, np.float32)
    tf = _dev(torch, f, 140, torch.float32)
    ax, ay = fvm.gradient_edges(tf, NLEV, averaged=True)
    dx, dy = fvm.gradient_edges(tf, NLEV)
    torch.cuda.synchronize()
    wx, wy = om.gradient(f, NLEV, nodes=nodes)
    vx, vy = om.gradient_averaged(f)
    vx, vy = vx[nodes], vy[nodes]
    pick = lambda t: t.index_select(0, idx)[:, :NLEV].double().cpu().numpy()
    err = {"difference.gx": _relmax(pick(dx), wx), "difference.gy": _relmax(pick(dy), wy),
           "averaged.gx": _relmax(pick(ax), vx), "averaged.gy": _relmax(pick(ay), vy)}
    REPORT["O%dx137 sampled edge-flux gradient fp32, difference vs averaged form" % N] = err
    _write_report()
    assert err["difference.gx"] <= 1e-5 and err["difference.gy"] <= 1e-5, err
    assert err["averaged.gx"] <= 2e-3 and err["averaged.gy"] <= 2e-3, err
    # the averaged form's FP32 error is the larger one (cancellation)
    assert max(err["averaged.gx"], err["averaged.gy"]) > max(err["difference.gx"], err["difference.gy"])


def test_averaged_flux_gradient_fp64_parity(torch, pfvm, omesh):
    fvm, om = pfvm(32), omesh(32)
    g = om.grid()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], 9)
    tf = _dev(torch, f, 10, torch.float64)
    ax, ay = fvm.gradient_edges(tf, 9, averaged=True)
    torch.cuda.synchronize()
    vx, vy = om.gradient_averaged(f)
    assert _relmax(ax[:, :9].cpu().numpy(), vx) <= 1e-13
    assert _relmax(ay[:, :9].cpu().numpy(), vy) <= 1e-13
