"""Autotuner of the launch shapes of the nabla kernels.

Every operator has two kernels whose results are bitwise equal: the
shared-memory node-group (tile) kernel, with the groups per tile and the
blocks per SM free (``atlas_fvm_set_group``), and the per-node kernel, with
five free parameters: levels per thread (``vec``), CSR entries per load
batch (``batch``), threads per block, blocks per SM and the length of the
item tile each block walks (``tile``, in passes of the block;
``atlas_fvm_set_launch``).  ``tune_fvm`` times each candidate of both with
CUDA events on the real field sizes and installs the fastest;
``tune_batch`` does the same for the tile size and block shape of a
persistent batched launch.  Results are cached in the JSON file named by
``ATLASGB_TUNE_CACHE`` (if set), keyed by device name, grid, dtype, level
count and leading dimension.
"""
from __future__ import annotations

import itertools
import json
import os

from . import atlas
from .capi import ATLAS_BF16, ATLAS_F32, ATLAS_F64

# The tile length applies to bfloat16 fields and to the FP32 Laplacian (node
# pairs); the other FP32 and FP64 kernels walk a grid-stride loop.
CANDIDATES = {
    ATLAS_F32: dict(vec=(4, 2), batch=(6, 3), threads=(128, 256, 512), bps=(0,), tile=(1, 8)),
    ATLAS_F64: dict(vec=(2, 1), batch=(6, 3), threads=(128, 256), bps=(0,), tile=(1,)),
    ATLAS_BF16: dict(vec=(8, 4), batch=(6, 3), threads=(128, 256), bps=(0,), tile=(1, 8, 64)),
}
# fields of this many levels or fewer run the one-ring operators on the
# per-node kernels unless the node-group kernels are forced (the library's
# rule; the Laplacian runs the node-group kernel at any level count)
TILE_MIN_LEVELS = {ATLAS_F32: 80, ATLAS_BF16: 96}
ONE_INPUT = ("gradient", "divergence_adjoint", "vector_gradient", "curl_adjoint")
# node-group (tile) kernel candidates: (groups per tile, blocks per SM, nodes per consumer warp,
# grid rows per tile)
# (more than eleven groups: the Laplacian only; other operators then run
# per node)
TILE_CANDIDATES = ((10, 1, 4, 2), (12, 1, 4, 2), (15, 1, 4, 1), (8, 1, 4, 2), (9, 1, 4, 3), (11, 1, 4, 1),
                   (7, 1, 4, 1), (4, 2, 4, 1), (7, 1, 2, 1))
_TORCH_DT = None


def tile_candidates(op, dtype=ATLAS_F32):
    """The node-group candidates that apply to op: tiles of more than eleven
    groups only where the kernel has the registers for them (the Laplacian;
    the one-input operators in bfloat16)."""
    big = op == "laplacian" or (dtype == ATLAS_BF16 and op in ONE_INPUT)
    return tuple(c for c in TILE_CANDIDATES if c[0] <= 11 or big)


def _torch_dtype(code):
    import torch
    return {ATLAS_F32: torch.float32, ATLAS_F64: torch.float64, ATLAS_BF16: torch.bfloat16}[code]


def _cache_path():
    return os.environ.get("ATLASGB_TUNE_CACHE")


def _load_cache():
    p = _cache_path()
    if p and os.path.exists(p):
        try:
            with open(p) as fh:
                return json.load(fh)
        except (OSError, ValueError):
            return {}
    return {}


def _store_cache(c):
    p = _cache_path()
    if not p:
        return
    tmp = p + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(c, fh, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _grid_key(grid):
    """Cache key of a grid: its family and size (O<N>, F<N>, or a regional
    projection with its points per row and rows)."""
    if grid.projection is not None:
        return "%s%dx%d" % (grid.projection, grid.nx, grid.ny)
    return ("F%d" if grid.regular else "O%d") % grid.N


def _call(fvm, op, ins, outs, nlev):
    if op == "gradient":
        fvm.gradient(ins[0], nlev, out=(outs[0], outs[1]))
    elif op == "divergence":
        fvm.divergence(ins[0], ins[1], nlev, out=outs[0])
    elif op == "laplacian":
        fvm.laplacian(ins[0], nlev, out=outs[0])
    elif op == "gradient_adjoint":
        fvm.gradient_adjoint(ins[0], ins[1], nlev, out=outs[0])
    elif op == "curl":
        fvm.curl(ins[0], ins[1], nlev, out=outs[0])
    elif op == "vector_gradient":
        fvm.vector_gradient(ins[0], ins[1], nlev, out=tuple(outs[:4]))
    else:
        fvm.divergence_adjoint(ins[0], nlev, out=(outs[0], outs[1]))


def time_call(fn, reps=5, warmup=2):
    """Average milliseconds of fn() over reps launches (CUDA events, current stream)."""
    import torch
    for _ in range(warmup):
        fn()
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune_fvm(fvm, dtype=ATLAS_F32, nlev=137, ld=None, ops=tuple(atlas.OPS), fields=None, reps=5, verbose=False):
    """Pick and install the fastest launch shape of every operator in ops.
    fields: optional (f, u, v) tensors [nnodes, ld] to time on (else zeros)."""
    import torch
    dev_name = torch.cuda.get_device_name()
    es = {ATLAS_F32: 4, ATLAS_F64: 8, ATLAS_BF16: 2}[dtype]
    if ld is None:
        q = 16 // es
        ld = (nlev + q - 1) // q * q
    key_base = "%s|%s|dt%d|L%d|ld%d" % (dev_name, _grid_key(fvm.grid), dtype, nlev, ld)
    cache = _load_cache()
    if fields is None:
        t = _torch_dtype(dtype)
        fields = [torch.randn((fvm.nnodes, ld), device="cuda").to(t) for _ in range(3)]
    outs = [torch.empty_like(fields[0]) for _ in range(4)]
    best = {}
    for op in ops:
        key = key_base + "|" + op
        if key in cache:
            c = cache[key]
            fvm.set_launch(op, c["vec"], c["batch"], c["threads"], c["bps"], c.get("tile", 1), dtype=dtype)
            if c.get("kernel", "node") == "tile":
                fvm.set_group(op, 1, c["tile_bps"], c["groups"], dtype=dtype, nodes_per_warp=c.get("npw", 4),
                              rows_per_tile=c.get("rows", 1))
            else:
                fvm.set_group(op, 0, dtype=dtype)
            best[op] = c
            continue
        ins = (fields[1], fields[2]) if op in ("divergence", "gradient_adjoint", "curl", "vector_gradient") \
            else (fields[0],)
        cand = CANDIDATES[dtype]
        results = []
        # the per-node kernel's shapes
        fvm.set_group(op, 0, dtype=dtype)
        for vec, batch, threads, bps, tile in itertools.product(cand["vec"], cand["batch"], cand["threads"],
                                                                cand["bps"], cand["tile"]):
            fvm.set_launch(op, vec, batch, threads, bps, tile, dtype=dtype)
            ms = time_call(lambda: _call(fvm, op, ins, outs, nlev), reps=reps)
            results.append((ms, "node", vec, batch, threads, bps, tile, 0, 0, 0, 0))
            if verbose:
                print("tune %-18s node vec=%d batch=%d threads=%d bps=%d tile=%d: %.4f ms" %
                      (op, vec, batch, threads, bps, tile, ms))
        _, _, vec, batch, threads, bps, tile, _, _, _, _ = min(results)
        fvm.set_launch(op, vec, batch, threads, bps, tile, dtype=dtype)
        # the tile kernel's shapes (where it applies to these fields: the
        # library runs it on fields of more than TILE_MIN_LEVELS levels)
        if (nlev > TILE_MIN_LEVELS.get(dtype, 96) or op == "laplacian") and \
                fvm.tile_info(op, nlev, ld, dtype)["stages"] > 0:
            for groups, tbps, npw, rows in tile_candidates(op, dtype):
                fvm.set_group(op, 1, tbps, groups, dtype=dtype, nodes_per_warp=npw, rows_per_tile=rows)
                ms = time_call(lambda: _call(fvm, op, ins, outs, nlev), reps=reps)
                results.append((ms, "tile", vec, batch, threads, bps, tile, groups, tbps, npw, rows))
                if verbose:
                    print("tune %-18s tile groups=%d bps=%d npw=%d rows=%d: %.4f ms" % (op, groups, tbps, npw, rows,
                                                                                      ms))
        ms, kernel, vec, batch, threads, bps, tile, groups, tbps, npw, rows = min(results)
        if kernel == "tile":
            fvm.set_group(op, 1, tbps, groups, dtype=dtype, nodes_per_warp=npw, rows_per_tile=rows)
        else:
            fvm.set_group(op, 0, dtype=dtype)
        # the launch shape the node-group kernel takes (blocks per SM may be
        # fewer than asked when shared memory or registers are short)
        shape = fvm.tile_info(op, nlev, ld, dtype) if kernel == "tile" else dict(blocks_per_sm=0, stages=0)
        best[op] = dict(kernel=kernel, vec=vec, batch=batch, threads=threads, bps=bps, tile=tile, groups=groups,
                        tile_bps=tbps, npw=npw, rows=rows, tile_blocks=shape["blocks_per_sm"],
                        tile_stages=shape["stages"], ms=ms,
                        sweep=[dict(ms=r[0], kernel=r[1], vec=r[2], batch=r[3], threads=r[4], bps=r[5], tile=r[6],
                                    groups=r[7], tile_bps=r[8], npw=r[9], rows=r[10]) for r in results])
        cache[key] = {k: best[op][k] for k in ("kernel", "vec", "batch", "threads", "bps", "tile", "groups",
                                              "tile_bps", "npw", "rows", "ms")}
    _store_cache(cache)
    return best


def tune_batch(make, candidates=None, reps=5, verbose=False):
    """make(tune_dict) -> Batch; returns (best Batch, best tune, sweep)."""
    if candidates is None:
        candidates = [dict(vec=4, tile_items=t, threads=th, blocks_per_sm=0, plain_waves=pw)
                      for t in (1024, 4096) for th in (128, 256) for pw in (-1, 1, 2, 4, 8)]
    sweep = []
    best = None
    for c in candidates:
        b = make(c)
        ms = time_call(b.launch, reps=reps)
        sweep.append(dict(ms=ms, **c))
        if verbose:
            print("tune batch %r: %.4f ms" % (c, ms))
        if best is None or ms < best[0]:
            if best is not None:
                best[1].close()
            best = (ms, b, c)
        else:
            b.close()
    return best[1], best[2], sweep
