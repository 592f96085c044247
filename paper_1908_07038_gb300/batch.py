"""Batched application of the operators to many fields in one persistent
launch (``atlas_batch_*``; the fields of ``plain_waves`` full GPU waves or
more -- four by default, none with -1 -- get plain launches of their own in
the same call), optionally captured once in a CUDA graph and replayed.

A ``Batch`` holds its descriptor table (passed whole to each launch as a
kernel parameter); the field pointers are fixed when it is created, which is
also what a CUDA graph needs.  ``plain``
runs the same work as one launch per field, for comparison.
"""
from __future__ import annotations

import ctypes

from . import capi
from .atlas import _dtype_code, _stream


class Batch:
    """One batched call over a list of (op, fvm, inputs, outputs) jobs.

    jobs: sequence of dicts with keys op ('gradient' | 'divergence'), fvm,
    ins (tuple of tensors), outs (tuple of tensors), nlev.
    """

    def __init__(self, jobs, tune=None):
        n = len(jobs)
        if n == 0:
            raise ValueError("a batch needs at least one job")
        arr = (capi.atlas_batch_desc * n)()
        dt = None
        for k, j in enumerate(jobs):
            d = arr[k]
            grad = j["op"] == "gradient"
            d.op = capi.ATLAS_OP_GRADIENT if grad else capi.ATLAS_OP_DIVERGENCE
            d.fvm = j["fvm"].handle.value
            t0 = j["ins"][0]
            d.in0 = t0.data_ptr()
            d.in1 = None if grad else j["ins"][1].data_ptr()
            d.out0 = j["outs"][0].data_ptr()
            d.out1 = j["outs"][1].data_ptr() if grad else None
            d.nlev = int(j["nlev"])
            d.ld = t0.stride(0)
            c = _dtype_code(t0)
            if dt is not None and c != dt:
                raise ValueError("all fields of a batch need one dtype")
            dt = c
        tn = None
        if tune:
            tn = capi.atlas_batch_tune(int(tune.get("vec", 0)), int(tune.get("tile_items", 0)),
                                       int(tune.get("threads", 0)), int(tune.get("blocks_per_sm", 0)),
                                       int(tune.get("plain_waves", 0)))
        h = ctypes.c_void_p()
        capi.atlas_batch_create(arr, n, dt, ctypes.byref(tn) if tn is not None else None, ctypes.byref(h))
        self.handle = h
        self.jobs = list(jobs)  # keeps the fields alive
        tiles, nl = ctypes.c_int64(), ctypes.c_int64()
        capi.atlas_batch_info(h, ctypes.byref(tiles), ctypes.byref(nl))
        self.tiles, self.node_levels = tiles.value, nl.value
        self.graph = None

    def launch(self, stream=None):
        capi.atlas_batch_launch(self.handle, _stream() if stream is None else stream)

    def capture(self):
        """Capture one launch in a CUDA graph (on a side stream, as torch requires)."""
        import torch
        self.launch()  # warm: module load outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.launch()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def close(self):
        if self.handle is not None and self.handle.value:
            capi.atlas_batch_destroy(self.handle)
        self.handle = None
        self.graph = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plain(jobs):
    """The same work as one kernel launch per field."""
    for j in jobs:
        fvm = j["fvm"]
        if j["op"] == "gradient":
            fvm.gradient(j["ins"][0], j["nlev"], out=tuple(j["outs"]))
        else:
            fvm.divergence(j["ins"][0], j["ins"][1], j["nlev"], out=j["outs"][0])


GRIDS = (80, 160, 320, 640)
LEVELS = (1, 60, 91, 137)


def make_jobs(fvms, nfields=24, seed=3, dtype=None, device="cuda"):
    """Seeded mixed batch: grid drawn from O80/O160/O320/O640, level count from
    {1, 60, 91, 137}, scalar fields to the gradient and vector fields to the
    divergence (alternating), FP32 by default.  fvms: dict N -> Fvm.
    Field values come from the synthetic recipe at each grid's nodes."""
    import numpy as np
    import torch

    import synthetic
    dtype = torch.float32 if dtype is None else dtype
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for k in range(nfields):
        N = int(GRIDS[rng.integers(len(GRIDS))])
        nlev = int(LEVELS[rng.integers(len(LEVELS))])
        fvm = fvms[N]
        g = fvm.grid.arrays()
        es = torch.tensor([], dtype=dtype).element_size()
        q = 16 // es
        ld = (nlev + q - 1) // q * q
        to = lambda x: torch.from_numpy(synthetic.padded(x, ld)).to(device=device, dtype=dtype)
        if k % 2 == 0:
            f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, seed=100 + k)
            tf = to(f)
            jobs.append(dict(op="gradient", fvm=fvm, ins=(tf,), outs=(torch.zeros_like(tf), torch.zeros_like(tf)),
                             nlev=nlev, N=N))
        else:
            u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, seeds=(200 + k, 300 + k), noise=True)
            tu, tv = to(u), to(v)
            jobs.append(dict(op="divergence", fvm=fvm, ins=(tu, tv), outs=(torch.zeros_like(tu),), nlev=nlev, N=N))
    return jobs
