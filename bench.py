"""Benchmark of the nabla operators on O1280 x 137 levels (one GB300).

One step = one pass of the whole operator set on one batch of synthetic
fields resident in HBM: gradient of f, divergence of (u, v), Laplacian of f,
gradient adjoint of (u, v) and divergence adjoint of f, each a single fused
node-stencil kernel, FP32 fields with FP64-built geometry.  The metric is
node-levels per second over the step (5 * nnodes * nlev per step), plus the
achieved fraction of the HBM roofline of the dominant kernel; the FP64 and
BF16-storage forms are timed in the same run and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun every rank runs an independent replica on its own GPU (the
operators need no exchange on one grid); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Nabla grad node-levels/s & % HBM roofline, FP32 vs FP64, O1280 x 137 levels"
N_GRID, NLEV = 1280, 137
OPS = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint")
# (inputs, outputs) per operator
IO = {"gradient": (1, 2), "divergence": (2, 1), "laplacian": (1, 1), "gradient_adjoint": (2, 1),
      "divergence_adjoint": (1, 2), "curl": (2, 1), "vector_gradient": (2, 4)}
# operators beyond the five of the step, timed on the same fields
MORE_OPS = ("curl", "vector_gradient")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(value, ws, device):
    """The largest of one float per rank (a job takes as long as its slowest
    rank); every rank gets it.  ws == 1 needs no process group."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank, ws, ms):
    """Whole-job throughput: the units all ranks processed over the time of the
    slowest rank (milliseconds)."""
    return ws * units_per_rank / (ms * 1e-3)


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_o1280.json")
KERNEL_SOURCES = tuple(os.path.join(ROOT, "paper_1908_07038_gb300", "csrc", f)
                       for f in ("kernels.cu", "group.cuh", "group.cu", "group_f32.cu", "bounds.cuh", "patterns.h"))


def _kernel_hash():
    """SHA-256 of the kernel sources, in order (the traffic capture is keyed
    to it)."""
    import hashlib
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(op):
    """DRAM bytes per launch of op from the committed ncu capture, or None when
    the kernels have changed since the counters were taken."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
        if d.get("kernels_sha256") != _kernel_hash():
            return None
        return float(d["per_launch_bytes"][op])
    except (OSError, ValueError, KeyError):
        return None


# kernels of the FP32 operators on 137 levels: the shared-memory node-group
# kernel <storage, inputs, outputs, B term, weights per entry, part A and
# part B levels per lane, steps per batch, nodes per consumer warp>, or the
# per-node kernel
TILE_KERNEL_BASE = {"gradient": "tile_kernel<float,1,2,0,2,4,1,2",
                    "divergence": "tile_kernel<float,2,1,1,2,4,1,2",
                    "laplacian": "tile_kernel<float,1,1,0,1,4,1,4",
                    "gradient_adjoint": "tile_kernel<float,2,1,1,2,4,1,2",
                    "divergence_adjoint": "tile_kernel<float,1,2,1,2,4,1,2"}
TILE_DEFAULT_NPW = {}


def _tile_kernel_name(op, npw=None):
    npw = TILE_DEFAULT_NPW.get(op, 4) if npw is None else npw
    return "%s,%d>" % (TILE_KERNEL_BASE[op], npw)


NODE_KERNEL_NAME = {"gradient": "stencil_kernel<float,float,1,2,4,0,0,B,1>",
                    "divergence": "stencil_kernel<float,float,2,1,4,1,0,B,1>",
                    "laplacian": "stencil_kernel<float,float,1,1,4,0,1,B,1>",
                    "gradient_adjoint": "stencil_kernel<float,float,2,1,4,1,0,B,1>",
                    "divergence_adjoint": "stencil_kernel<float,float,1,2,4,1,0,B,1>"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _fields_torch(torch, lon, lat, nlev, ld, dtype, device, seed):
    """Synthetic fields of the standard recipe (base field scaled by
    1 + 0.01 k plus N(0, 1e-3^2) noise) generated on the device with a seeded
    torch generator, stored [node][ld] with zero padding."""
    import synthetic
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    lon_t = torch.from_numpy(lon).to(device)
    lat_t = torch.from_numpy(lat).to(device)
    scale = 1.0 + 0.01 * torch.arange(nlev, device=device, dtype=torch.float64)
    bs = torch.from_numpy(synthetic.base_scalar(lon, lat)).to(device)
    bu, bv = (torch.from_numpy(x).to(device) for x in synthetic.base_vector(lon, lat))
    del lon_t, lat_t
    out = []
    for base in (bs, bu, bv):
        t = torch.zeros((base.shape[0], ld), dtype=dtype, device=device)
        V = base.shape[0]
        step = 1 << 20
        for i0 in range(0, V, step):
            i1 = min(V, i0 + step)
            blk = base[i0:i1, None] * scale[None, :]
            blk = blk + synthetic.NOISE_SIGMA * torch.randn((i1 - i0, nlev), generator=g, device=device,
                                                            dtype=torch.float64)
            t[i0:i1, :nlev] = blk.to(dtype)
        out.append(t)
    return out


def _run_step(fvm, f, u, v, outs, nlev):
    gx, gy, d, lap, ga, du, dv = outs
    fvm.gradient(f, nlev, out=(gx, gy))
    fvm.divergence(u, v, nlev, out=d)
    fvm.laplacian(f, nlev, out=lap)
    fvm.gradient_adjoint(u, v, nlev, out=ga)
    fvm.divergence_adjoint(f, nlev, out=(du, dv))


def _time_ops(torch, fvm, f, u, v, outs, nlev, steps, warmup, barrier):
    """Warm up, then time `steps` steps with CUDA events on the launching
    stream: whole-step time and per-operator kernel time."""
    gx, gy, d, lap, ga, du, dv = outs
    calls = [lambda: fvm.gradient(f, nlev, out=(gx, gy)), lambda: fvm.divergence(u, v, nlev, out=d),
             lambda: fvm.laplacian(f, nlev, out=lap), lambda: fvm.gradient_adjoint(u, v, nlev, out=ga),
             lambda: fvm.divergence_adjoint(f, nlev, out=(du, dv))]
    for _ in range(warmup):
        for c in calls:
            c()
    stream = torch.cuda.current_stream()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(steps)]
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(steps):
        ev[s][0].record(stream)
        for k, c in enumerate(calls):
            c()
            ev[s][k + 1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    total_ms = t0.elapsed_time(t1)
    per_op = [0.0] * len(calls)
    for s in range(steps):
        for k in range(len(calls)):
            per_op[k] += ev[s][k].elapsed_time(ev[s][k + 1])
    return total_ms, [p / steps for p in per_op]


def _alg_bytes(op, V, nlev, esize, table_bytes):
    nin, nout = IO[op]
    return (nin + nout) * V * nlev * esize + table_bytes


_NNZ = {}


def _table_bytes(fvm, op, wbytes):
    if op not in _NNZ:
        _NNZ[op] = fvm.stencil_table(op)["nbr"].shape[0]
    return _table_bytes_nnz(fvm, op, wbytes, _NNZ[op])


def _table_bytes_of(fvm, op, wbytes):
    """_table_bytes for an fvm other than the benchmark's (no caching)."""
    return _table_bytes_nnz(fvm, op, wbytes, fvm.stencil_table(op)["nbr"].shape[0])


def _table_bytes_nnz(fvm, op, wbytes, nnz):
    V = fvm.nnodes
    has_b = op in ("divergence", "gradient_adjoint", "divergence_adjoint", "curl", "vector_gradient")
    nw = 1 if op == "laplacian" else 2
    return 4 * (V + 1) + nnz * (4 + nw * wbytes) + (2 * wbytes * V if has_b else 0)


# Nominal FP64 rate of a GB300 at its maximum SM clock (2070 MHz), for
# context; the FP64 roofline is quoted against the rate the library's FP64
# FMA kernel measures in the same run (atlas.measure_fp64_rate).
FP64_NOMINAL_TFLOPS, SM_MAX_MHZ = 1.25, 2070.0


def _fp64_flops(fvm, op, nlev):
    """Algorithmic FP64 flops of one launch (an FMA counts 2), the arithmetic
    of the operator's node formula as the method writes it: each stencil
    term w (x_j - x_i) of every output costs one subtraction per input and
    one multiply-add per (input, output) weight, and the per-node B term one
    multiply-add per (input, output) pair."""
    if op not in _NNZ:
        _NNZ[op] = fvm.stencil_table(op)["nbr"].shape[0]
    nnz, V = _NNZ[op], fvm.nnodes
    per_entry = {"gradient": 1 + 2 * 2, "divergence_adjoint": 1 + 2 * 2, "laplacian": 1 + 2,
                 "divergence": 2 + 2 * 2, "gradient_adjoint": 2 + 2 * 2}[op]
    per_node = {"gradient": 0, "laplacian": 0, "divergence_adjoint": 2 * 2, "divergence": 2 * 2,
                "gradient_adjoint": 2 * 2}[op]
    return (nnz * per_entry + V * per_node) * nlev


def _precision(torch, fvm, lon, lat, nlev, seed):
    """Error of the FP32 and BF16-storage paths against the FP64 path on the
    whole field: max |x - x64| / max |x64| per operator (worst output
    component), over all nodes and levels.  The FP64 path (pinned to the FP64
    oracle at 1e-13) stands in for the oracle at this size; each path's FP64
    reference runs on the same rounded inputs, so the figure is the
    arithmetic's error, not the inputs' rounding."""
    ops = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint", "curl", "vector_gradient",
           "curl_adjoint")
    nin = {"divergence": 2, "gradient_adjoint": 2, "curl": 2, "vector_gradient": 2}

    def run(op, a, b):
        if op == "gradient":
            return fvm.gradient(a, nlev)
        if op == "laplacian":
            return (fvm.laplacian(a, nlev),)
        if op == "divergence_adjoint":
            return fvm.divergence_adjoint(a, nlev)
        if op == "curl_adjoint":
            return fvm.curl_adjoint(a, nlev)
        if op == "vector_gradient":
            return fvm.vector_gradient(a, b, nlev)
        return (getattr(fvm, op)(a, b, nlev),)

    def relmax(x, ref):
        den = ref.abs().max().item()
        return (x[:, :nlev].double() - ref[:, :nlev]).abs().max().item() / (den if den > 0 else 1.0)

    f64, u64, v64 = _fields_torch(torch, lon, lat, nlev, 138, torch.float64, "cuda", seed)
    out = {}
    for name, dt, ldx in (("fp32", torch.float32, 140), ("bf16", torch.bfloat16, 144)):
        out[name] = {}
        for op in ops:
            a = f64 if nin.get(op, 1) == 1 else u64
            b = v64
            ar = torch.zeros((a.shape[0], ldx), dtype=dt, device="cuda")
            br = torch.zeros((a.shape[0], ldx), dtype=dt, device="cuda")
            ar[:, :nlev] = a[:, :nlev].to(dt)
            br[:, :nlev] = b[:, :nlev].to(dt)
            a64 = torch.zeros((a.shape[0], 138), dtype=torch.float64, device="cuda")
            b64 = torch.zeros((a.shape[0], 138), dtype=torch.float64, device="cuda")
            a64[:, :nlev] = ar[:, :nlev].double()
            b64[:, :nlev] = br[:, :nlev].double()
            ref = run(op, a64, b64)
            got = run(op, ar, br)
            out[name][op] = float("%.3g" % max(relmax(x, r) for x, r in zip(got, ref)))
            del ar, br, a64, b64, ref, got
    del f64, u64, v64
    torch.cuda.empty_cache()
    return out


def _shape(t):
    """The launch shape the tuner picked, as a short string."""
    if t.get("kernel") == "tile":
        if "tile_blocks" in t:
            return "tile kernel, %d groups per tile over %d grid row(s), %d node(s) per warp, %d block(s) of %d " \
                "stages per SM" % (t["groups"], t.get("rows", 1), t.get("npw", 4), t["tile_blocks"], t["tile_stages"])
        return "tile kernel, %d groups per tile, %d block(s) per SM asked" % (t["groups"], t["tile_bps"])
    return "per-node kernel, vec %d, batch %d, %d threads, tile %d" % (t["vec"], t["batch"], t["threads"],
                                                                       t.get("tile", 1))


def _cpu_baseline(grid, fvm_nodes, f_host, u_host, v_host, nlev, budget_s=30.0):
    """The oracle as it stands, single-threaded, on a contiguous node sample
    of the same workload (all five operators)."""
    from oracle.oracle import Mesh
    om = Mesh(grid)
    n = 64
    while True:
        nodes = np.arange(0, n, dtype=np.int64) + fvm_nodes // 3
        t = time.perf_counter()
        om.gradient(f_host, nlev, nodes=nodes)
        om.divergence(u_host, v_host, nlev, nodes=nodes)
        om.laplacian(f_host, nlev, nodes=nodes)
        om.gradient_adjoint(u_host, v_host, nlev, nodes=nodes)
        om.divergence_adjoint(f_host, nlev, nodes=nodes)
        dt = time.perf_counter() - t
        if dt > budget_s / 4 or n >= fvm_nodes:
            break
        n = min(fvm_nodes, int(n * max(2.0, budget_s / max(dt, 1e-3) / 2)))
    value = 5 * n * nlev / dt
    return {"value": value, "unit": "node-levels/s", "cores": 1, "kind": "oracle",
            "sample": "nodes %d..%d of O1280 (%d nodes) x %d levels, all five operators, %.1f s" %
                      (int(nodes[0]), int(nodes[-1]), n, nlev, dt)}


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_1908_07038_gb300 import atlas

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    nlev = NLEV
    fvm = atlas.build_fvm(args.grid)
    V = fvm.nnodes
    g = fvm.grid.arrays()
    fvm.prepare(OPS, dtypes=(atlas.ATLAS_F32, atlas.ATLAS_F64, atlas.ATLAS_BF16))
    if not args.no_more:
        fvm.prepare(MORE_OPS, dtypes=(atlas.ATLAS_F32,))
    hbm, peak_kind = _peaks()

    # ------------------------------------------------------------ FP32 main
    from paper_1908_07038_gb300 import tune
    ld = 140
    f, u, v = _fields_torch(torch, g["lon"], g["lat_node"], nlev, ld, torch.float32, "cuda", 1234 + rank)
    outs = [torch.empty_like(f) for _ in range(7)]
    tuned = {} if args.no_tune else tune.tune_fvm(fvm, atlas.ATLAS_F32, nlev, ld, OPS, fields=(f, u, v), reps=3)
    for op, t in tuned.items():
        print("tuned %s: %s (%.3f ms)" % (op, _shape(t), t["ms"]), file=sys.stderr)
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, per_op = _time_ops(torch, fvm, f, u, v, outs, nlev, args.steps, args.warmup, barrier)
    clocks = sampler.stop()
    total_ms = _max_over_ranks(total_ms, ws, "cuda")
    ms_step = total_ms / args.steps
    node_levels_step = 5 * V * nlev
    value = _job_rate(node_levels_step, ws, ms_step)

    # per-op roofline (algorithmic bytes / average kernel time)
    tables = {op: _table_bytes(fvm, op, 4) for op in OPS}
    per = {}
    for op, ms in zip(OPS, per_op):
        b = _alg_bytes(op, V, nlev, 4, tables[op])
        per[op] = {"ms": round(ms, 4), "node_levels_per_s": V * nlev / (ms * 1e-3),
                   "alg_bytes": b, "gbs": b / (ms * 1e-3) / 1e9, "frac": b / (ms * 1e-3) / 1e9 / hbm}
    dom = max(OPS, key=lambda o: per[o]["ms"])
    traffic = _traffic(dom) if args.grid == N_GRID else None
    dom_t = tuned.get(dom, {})
    dom_name = _tile_kernel_name(dom, dom_t.get("npw")) if dom_t.get("kernel", "tile") == "tile" else NODE_KERNEL_NAME[dom]
    roofline = {"bound": "hbm", "kernel": dom_name, "operator": dom,
                "achieved": round(per[dom]["gbs"], 1),
                "peak": hbm, "unit": "GB/s", "frac": round(per[dom]["frac"], 4),
                "traffic": traffic, "traffic_gbs": round(traffic / (per[dom]["ms"] * 1e-3) / 1e9, 1) if traffic else None,
                "peak_kind": peak_kind}

    # ------------------------------------------- curl and vector gradient
    more = {}
    if not args.no_more:
        mt = {} if args.no_tune else tune.tune_fvm(fvm, atlas.ATLAS_F32, nlev, ld, MORE_OPS, fields=(f, u, v), reps=3)
        calls = {"curl": lambda: fvm.curl(u, v, nlev, out=outs[0]),
                 "vector_gradient": lambda: fvm.vector_gradient(u, v, nlev, out=tuple(outs[:4]))}
        for op in MORE_OPS:
            ms = _max_over_ranks(tune.time_call(calls[op], reps=max(5, args.steps), warmup=args.warmup), ws, "cuda")
            # the vector gradient reads its table once per component
            tb = _table_bytes(fvm, op, 4) * (2 if op == "vector_gradient" else 1)
            b = _alg_bytes(op, V, nlev, 4, tb)
            more[op] = {"ms": round(ms, 4), "node_levels_per_s": _job_rate(V * nlev, ws, ms),
                        "alg_bytes": b, "frac_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4),
                        "launches": 2 if op == "vector_gradient" else 1,
                        "tuned": _shape(mt[op]) if op in mt else None}
        # FP64 volume-weighted sums of one FP32 field (the conservation sums)
        iw = torch.empty(max(atlas.capi.atlas_fvm_integral_workspace_bytes(fvm.handle, nlev) // 8, 1),
                         dtype=torch.float64, device="cuda")
        io = torch.empty(nlev, dtype=torch.float64, device="cuda")
        ms = _max_over_ranks(tune.time_call(lambda: fvm.integral(f, nlev, out=io, ws=iw), reps=max(5, args.steps),
                                            warmup=args.warmup), ws, "cuda")
        b = V * nlev * 4 + V * 8
        fl = 2.0 * V * nlev
        more["integral_fp64"] = {"ms": round(ms, 4), "node_levels_per_s": _job_rate(V * nlev, ws, ms),
                                 "alg_bytes": b, "frac_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4),
                                 "fp64_tflops": round(fl / (ms * 1e-3) / 1e12, 3),
                                 "launches": 2}
        del iw, io
        # the edge-based two-pass forms: edge fluxes through a workspace
        # (E x ld per flux component), then the signed node gather
        wsz = max(atlas.capi.atlas_nabla_workspace_bytes(fvm.handle, atlas.OPS[o], 0, ld, atlas.ATLAS_F32)
                  for o in ("gradient", "divergence", "laplacian"))
        ew = torch.empty(wsz, dtype=torch.uint8, device="cuda")
        ecalls = (("gradient", lambda: fvm.gradient_edges(f, nlev, ws=ew, out=(outs[0], outs[1]))),
                  ("divergence", lambda: fvm.divergence_edges(u, v, nlev, ws=ew, out=outs[0])),
                  ("laplacian", lambda: fvm.laplacian_edges(f, nlev, ws=ew, out=outs[0])))
        for op, call in ecalls:
            ms = _max_over_ranks(tune.time_call(call, reps=max(5, args.steps), warmup=args.warmup), ws, "cuda")
            b = _alg_bytes(op, V, nlev, 4, 0)
            more[op + "_edges"] = {"ms": round(ms, 4), "node_levels_per_s": _job_rate(V * nlev, ws, ms),
                                   "alg_field_bytes": b, "frac_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4),
                                   "launches": 4 if op == "laplacian" else 2}
        del ew
        # remapping to the regular Gaussian grid of half the resolution
        M = args.grid // 2
        rm = atlas.Remap(fvm.mesh, atlas.Grid(M, regular=True))
        rn, _ = rm.tables()
        dst = torch.empty((rm.ntgt, ld), device="cuda")
        ms = _max_over_ranks(tune.time_call(lambda: rm.apply(f, nlev, out=dst), reps=max(5, args.steps),
                                            warmup=args.warmup), ws, "cuda")
        used = int(np.unique(rn).size)  # source rows the targets read
        b = (used + rm.ntgt) * nlev * 4 + rm.ntgt * 32
        more["remap_to_F%d" % M] = {"ms": round(ms, 4), "target_levels_per_s": _job_rate(rm.ntgt * nlev, ws, ms),
                                    "targets": rm.ntgt, "source_rows_read": used, "alg_bytes": b,
                                    "frac_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4), "launches": 1}
        del dst, rm
        # the regular Gaussian grid of the same latitudes (F<N/2>, 8 (N/2)^2 nodes)
        ff = atlas.build_fvm(M, regular=True)
        ff.prepare(("gradient", "laplacian"), dtypes=(atlas.ATLAS_F32,))
        Vf = ff.nnodes
        xf = torch.randn((Vf, ld), device="cuda")
        of = [torch.empty_like(xf) for _ in range(2)]
        if not args.no_tune:
            tune.tune_fvm(ff, atlas.ATLAS_F32, nlev, ld, ("gradient", "laplacian"), fields=(xf, xf, xf), reps=3)
        for op, call in (("gradient", lambda: ff.gradient(xf, nlev, out=(of[0], of[1]))),
                         ("laplacian", lambda: ff.laplacian(xf, nlev, out=of[0]))):
            ms = _max_over_ranks(tune.time_call(call, reps=max(5, args.steps), warmup=args.warmup), ws, "cuda")
            b = _alg_bytes(op, Vf, nlev, 4, _table_bytes_of(ff, op, 4))
            more["%s_F%d" % (op, M)] = {"ms": round(ms, 4), "node_levels_per_s": _job_rate(Vf * nlev, ws, ms),
                                        "nodes": Vf, "alg_bytes": b, "frac_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4)}
        del xf, of, ff
        # a limited-area configuration: 1536 x 1440 points at 2.5 km on a
        # Lambert conformal cone, 90 levels, same kernels with the regional tables
        from synthetic.regional import LAM, LAM_NLEV, LAM_NX, LAM_NY
        rf = atlas.build_fvm_regional(LAM[0], LAM_NX, LAM_NY, **LAM[1])
        rops = ("gradient", "divergence", "laplacian", "curl")
        rf.prepare(rops, dtypes=(atlas.ATLAS_F32,))
        Vr, lr, ldr = rf.nnodes, LAM_NLEV, 92
        xr, yr = (torch.randn((Vr, ldr), device="cuda") for _ in range(2))
        orr = [torch.empty_like(xr) for _ in range(2)]
        if not args.no_tune:
            tune.tune_fvm(rf, atlas.ATLAS_F32, lr, ldr, rops, fields=(xr, xr, yr), reps=3)
        rcalls = {"gradient": lambda: rf.gradient(xr, lr, out=(orr[0], orr[1])),
                  "divergence": lambda: rf.divergence(xr, yr, lr, out=orr[0]),
                  "laplacian": lambda: rf.laplacian(xr, lr, out=orr[0]),
                  "curl": lambda: rf.curl(xr, yr, lr, out=orr[0])}
        reg = {"grid": "Lambert conformal %dx%d, %d levels" % (LAM_NX, LAM_NY, lr), "nodes": Vr}
        for op in rops:
            ms = _max_over_ranks(tune.time_call(rcalls[op], reps=max(5, args.steps), warmup=args.warmup), ws, "cuda")
            b = _alg_bytes(op, Vr, lr, 4, _table_bytes_of(rf, op, 4))
            reg[op] = {"ms": round(ms, 4), "node_levels_per_s": _job_rate(Vr * lr, ws, ms), "alg_bytes": b,
                       "frac_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4)}
        more["regional_lambert"] = reg
        del xr, yr, orr, rf

    # ---------------------------------------------------------------- e2e
    # Host-resident fields through the public API: every step copies f, u, v
    # from pinned host memory and the seven results back (HostStep pipelines
    # the copies against the kernels on three streams).  The serial form
    # (copy in, compute, copy out on one stream) is timed beside it.
    e2e = None
    if not args.no_e2e:
        from paper_1908_07038_gb300.hoststep import HostStep
        hin = {n: t.cpu().pin_memory() for n, t in zip(("f", "u", "v"), (f, u, v))}
        hs = HostStep(fvm, nlev, ld, torch.float32)
        hout = {n: torch.empty(hs.dev[n].shape, dtype=torch.float32, pin_memory=True) for n in hs.outputs}
        stream = torch.cuda.current_stream()
        ksteps = max(2, min(args.steps, 5))
        hs.run(hin, hout)
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hs.begin(stream)
        for _ in range(ksteps):
            hs.enqueue(hin, hout)
        hs.join(stream)
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        e_ms = _max_over_ranks(a.elapsed_time(b) / ksteps, ws, "cuda")
        # the serial form on one stream
        nbytes = hs.nbytes
        sout = [hout[n] for n in ("gx", "gy", "div", "lap", "ga", "du", "dv")]

        def serial_step():
            for n, dv in zip(("f", "u", "v"), (f, u, v)):
                atlas.field_sync(dv.data_ptr(), hin[n].data_ptr(), nbytes, 0)
            _run_step(fvm, f, u, v, outs, nlev)
            for h, dv in zip(sout, outs):
                atlas.field_sync(h.data_ptr(), dv.data_ptr(), nbytes, 1)

        serial_step()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(2):
            serial_step()
        b.record(stream)
        torch.cuda.synchronize()
        s_ms = a.elapsed_time(b) / 2
        e2e = {"value": _job_rate(node_levels_step, ws, e_ms), "unit": "node-levels/s",
               "h2d_bytes_per_step": hs.h2d_bytes, "d2h_bytes_per_step": hs.d2h_bytes, "ms_per_step": round(e_ms, 3),
               "steps": ksteps, "link_gbs": round((hs.h2d_bytes + hs.d2h_bytes) / (e_ms * 1e-3) / 1e9, 1),
               "pipelined": True, "serial_ms_per_step": round(s_ms, 3)}
        del hin, hout, hs, sout

    # ------------------------------------------------ FP64 and BF16 beside
    side = {}
    if not args.no_side:
        f_host = f[:, :nlev].cpu().numpy() if rank == 0 and not args.no_cpu_baseline else None
        u_host = u[:, :nlev].cpu().numpy() if f_host is not None else None
        v_host = v[:, :nlev].cpu().numpy() if f_host is not None else None
        del f, u, v, outs
        torch.cuda.empty_cache()
        fp64_rate = atlas.measure_fp64_rate()  # TFLOP/s of dependent FP64 FMAs on every SM
        for name, dt, ldx, es, wb in (("fp64", torch.float64, 138, 8, 8), ("bf16", torch.bfloat16, 144, 2, 4)):
            fx, ux, vx = _fields_torch(torch, g["lon"], g["lat_node"], nlev, ldx, dt, "cuda", 99 + rank)
            ox = [torch.empty_like(fx) for _ in range(7)]
            code = atlas.ATLAS_F64 if name == "fp64" else atlas.ATLAS_BF16
            if not args.no_tune:
                tune.tune_fvm(fvm, code, nlev, ldx, OPS, fields=(fx, ux, vx), reps=2)
            k = max(3, args.steps // 4)
            tms, pops = _time_ops(torch, fvm, fx, ux, vx, ox, nlev, k, 3, barrier)
            entry = {"ms_per_step": round(tms / k, 4), "node_levels_per_s": node_levels_step / (tms / k * 1e-3),
                     "per_op": {}}
            for op, ms in zip(OPS, pops):
                bytes_ = _alg_bytes(op, V, nlev, es, _table_bytes(fvm, op, wb) if name == "fp64" else tables[op])
                entry["per_op"][op] = {"ms": round(ms, 4), "node_levels_per_s": V * nlev / (ms * 1e-3),
                                       "frac_hbm": round(bytes_ / (ms * 1e-3) / 1e9 / hbm, 4)}
                if name == "fp64":
                    tf = _fp64_flops(fvm, op, nlev) / (ms * 1e-3) / 1e12
                    entry["per_op"][op]["fp64_tflops"] = round(tf, 4)
                    entry["per_op"][op]["frac_fp64"] = round(tf / fp64_rate, 4)
            if name == "fp64":
                dom = max(OPS, key=lambda o: entry["per_op"][o]["ms"])
                entry["roofline"] = {"bound": "alu", "operator": dom,
                                     "achieved": entry["per_op"][dom]["fp64_tflops"], "peak": round(fp64_rate, 4),
                                     "unit": "TFLOP/s", "frac": entry["per_op"][dom]["frac_fp64"],
                                     "peak_kind": "measured",
                                     "peak_source": "the library's dependent FP64 FMA kernel on every SM, this run",
                                     "nominal": FP64_NOMINAL_TFLOPS}
            side[name] = entry
            del fx, ux, vx, ox
            torch.cuda.empty_cache()
    else:
        f_host = None

    # ------------------- FP32 and BF16 error against the FP64 path, whole field
    precision = None
    if not args.no_precision:
        precision = _precision(torch, fvm, g["lon"], g["lat_node"], nlev, 7 + rank)

    # ------------------------------------- 24 mixed fields, one launch each vs batched
    batched = None
    if not args.no_batch:
        from paper_1908_07038_gb300 import batch as B
        fvms = {N: atlas.build_fvm(N) for N in B.GRIDS}
        jobs = B.make_jobs(fvms, 24, seed=3)
        for N, fv in fvms.items():
            fv.prepare(("gradient", "divergence"), dtypes=(atlas.ATLAS_F32,))
            tune.tune_fvm(fv, atlas.ATLAS_F32, 137, 140, ("gradient", "divergence"), reps=2)

        def graph_ms(cfg):
            bb = B.Batch(jobs, tune=cfg)
            bb.capture()
            ms = tune.time_call(bb.replay, reps=20, warmup=3)
            n = bb.node_levels
            bb.close()
            return ms, n

        # the library's default split (fields of four waves and more in plain
        # launches of their own, the rest in one persistent launch), the
        # tuned split, and every field in the persistent launch
        ms_default, nl = graph_ms(None)
        bt, bt_cfg, _ = tune.tune_batch(lambda c: B.Batch(jobs, tune=c), reps=5)
        bt.close()
        ms_tuned, _ = graph_ms(bt_cfg)
        ms_persistent, _ = graph_ms(dict(bt_cfg, plain_waves=-1))
        ms_plain = tune.time_call(lambda: B.plain(jobs), reps=20, warmup=3)
        batched = {"fields": len(jobs), "node_levels": nl, "graph_replay_ms": round(ms_default, 4),
                   "config": "library default (plain_waves 4)",
                   "plain_launches_ms": round(ms_plain, 4),
                   "graph_node_levels_per_s": nl / (ms_default * 1e-3),
                   "plain_node_levels_per_s": nl / (ms_plain * 1e-3),
                   "tuned_graph_replay_ms": round(ms_tuned, 4), "tune": bt_cfg,
                   "all_persistent_graph_replay_ms": round(ms_persistent, 4),
                   "grids": sorted({j["N"] for j in jobs}), "levels": sorted({j["nlev"] for j in jobs})}
        del jobs, fvms
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and f_host is not None:
        cpu = _cpu_baseline(args.grid, V, f_host, u_host, v_host, nlev)

    if ws > 1:
        dist.barrier()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "node-levels/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "O%d octahedral grid (%d nodes, %d edges) x %d levels, field[node][ld=%d] FP32, "
                               "FP64-built geometry; step = gradient + divergence + Laplacian + gradient adjoint "
                               "+ divergence adjoint" % (args.grid, V, fvm.mesh.nedges, nlev, ld),
                   "l2": "inputs larger than L2 (%.2f GB per field, L2 129 MB), no flush" % (V * ld * 4 / 1e9), "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roofline, "per_op": {k: {"ms": v_["ms"], "node_levels_per_s": v_["node_levels_per_s"],
                                             "frac_hbm": round(v_["frac"], 4)} for k, v_ in per.items()},
        "more_ops": more,
        "side_by_side": side, "precision_vs_fp64": precision, "batched": batched,
        "tuned": {k: _shape(t) for k, t in tuned.items()},
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
        "gpu_launches": 5 * args.steps,
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on a bounded node sample of the same
    workload; rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import synthetic
    from oracle.oracle import Mesh
    om = Mesh(N_GRID)
    g = om.grid()
    nlev = NLEV
    # fields on a band of rows around the sample (the operators need the 2-ring)
    off = np.concatenate([[0], np.cumsum(g["pl"])])
    r0 = N_GRID // 2
    lo, hi = off[r0 - 3], off[r0 + 4]
    f = np.zeros((om.nnodes, nlev), np.float32)
    u = np.zeros_like(f)
    v = np.zeros_like(f)
    sl = slice(lo, hi)
    f[sl] = synthetic.level_scalar(g["lon"][sl], g["lat_node"][sl], nlev, np.float32)
    u[sl], v[sl] = synthetic.level_vector(g["lon"][sl], g["lat_node"][sl], nlev, np.float32)
    budget = float(os.environ.get("ORACLE_STEP_SECONDS", "2"))
    n = 16
    base = off[r0]
    while True:
        nodes = np.arange(base, base + n, dtype=np.int64)
        t = time.perf_counter()
        for _ in range(1):
            om.gradient(f, nlev, nodes=nodes)
            om.divergence(u, v, nlev, nodes=nodes)
            om.laplacian(f, nlev, nodes=nodes)
            om.gradient_adjoint(u, v, nlev, nodes=nodes)
            om.divergence_adjoint(f, nlev, nodes=nodes)
        dt = time.perf_counter() - t
        if dt > budget / 4 or n >= g["pl"][r0]:
            break
        n = min(int(g["pl"][r0]), int(n * max(2.0, budget / max(dt, 1e-3) / 2)))
    for _ in range(args.warmup):
        om.gradient(f, nlev, nodes=nodes)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        om.gradient(f, nlev, nodes=nodes)
        om.divergence(u, v, nlev, nodes=nodes)
        om.laplacian(f, nlev, nodes=nodes)
        om.gradient_adjoint(u, v, nlev, nodes=nodes)
        om.divergence_adjoint(f, nlev, nodes=nodes)
    el = time.perf_counter() - t0
    value = 5 * n * nlev * args.steps / el
    sample = "%d nodes of row %d of O1280 x %d levels per step, all five operators" % (n, r0, nlev)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "node-levels/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "O1280 octahedral grid x 137 levels (node sample), FP32 fields upcast to FP64"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value, "unit": "node-levels/s"},
            "e2e": {"value": value, "unit": "node-levels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP32/BF16 error against the FP64 path")
    ap.add_argument("--no-more", action="store_true", help="skip the curl and vector-gradient timings")
    ap.add_argument("--no-tune", action="store_true", help="library default launch shapes (profiling runs)")
    ap.add_argument("--grid", type=int, default=N_GRID,
                    help="octahedral number of a smaller case (profiling only; the metric is O1280)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
