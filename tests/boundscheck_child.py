"""Child process of test_gpu_boundscheck.py (not a test module).

Run with ATLASGB_BOUNDSCHECK=1: the package then loads the bounds-checked
build of the library, whose kernels check every index they take from a
table.  On O2 and O4 every kind of launch runs once -- the per-node and the
node-group (tile) stencil kernels (one or two consumer warps per group) for
every operator, FP64 and FP32, the
edge-based two-pass forms, a batched launch, band partitions and a remap --
and is compared with the FP64 oracle.  Any bounds violation makes the call
raise (ATLAS_EBOUNDS).  Prints one JSON line: the library's info string, the
number of comparisons, the worst relative error per precision and the
tile kernels' status word.
"""
import json
import sys

import numpy as np
import torch

import synthetic
from oracle.oracle import Mesh as OracleMesh
from paper_1908_07038_gb300 import atlas, batch, partition

OPS = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint", "curl", "vector_gradient",
       "curl_adjoint")
TWO_IN = ("divergence", "gradient_adjoint", "curl", "vector_gradient")


def relmax(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def gpu_op(fvm, op, x, y, nlev):
    if op == "gradient":
        return fvm.gradient(x, nlev)
    if op == "laplacian":
        return (fvm.laplacian(x, nlev),)
    if op == "divergence_adjoint":
        return fvm.divergence_adjoint(x, nlev)
    if op == "curl_adjoint":
        return fvm.curl_adjoint(x, nlev)
    if op == "vector_gradient":
        return fvm.vector_gradient(x, y, nlev)
    return (getattr(fvm, op)(x, y, nlev),)


def oracle_op(om, op, x, y, nlev):
    if op in TWO_IN:
        r = getattr(om, op)(x, y, nlev)
    else:
        r = getattr(om, op)(x, nlev)
    return r if isinstance(r, tuple) else (r,)


def main():
    worst = {"f64": 0.0, "f32": 0.0}
    tol = {"f64": 1e-13, "f32": 1e-5}
    cases = 0
    for N in (2, 4):
        fvm, om = atlas.build_fvm(N), OracleMesh(N)
        g = om.grid()
        lon, lat = g["lon"], g["lat_node"]
        for name, dt, ld in (("f64", torch.float64, 10), ("f32", torch.float32, 12)):
            nlev = 9
            f = synthetic.level_scalar(lon, lat, nlev)
            u, v = synthetic.level_vector(lon, lat, nlev)
            if name == "f32":  # the oracle is fed the same rounded inputs
                f, u, v = (a.astype(np.float32).astype(np.float64) for a in (f, u, v))
            dev = lambda a: torch.from_numpy(synthetic.padded(a, ld)).to(device="cuda", dtype=dt)
            fd, ud, vd = dev(f), dev(u), dev(v)
            for op in OPS:
                x, y = (ud, vd) if op in TWO_IN else (fd, None)
                want = oracle_op(om, op, u if op in TWO_IN else f, v, nlev)
                # per-node kernel; node-group kernels (FP32/BF16 fields) with one or two warps per group
                for group, npw in (((0, 4), (2, 4), (2, 2)) if name == "f32" else ((0, 4),)):
                    fvm.set_group(op, enable=group, nodes_per_warp=npw)
                    got = gpu_op(fvm, op, x, y, nlev)
                    torch.cuda.synchronize()
                    for a, b in zip(got, want):
                        e = relmax(a[:, :nlev].double().cpu().numpy(), b)
                        assert e <= tol[name], (N, name, op, group, e)
                        worst[name] = max(worst[name], e)
                        cases += 1
                fvm.set_group(op, enable=1, nodes_per_warp=4)
            # edge-based two-pass forms
            gx, gy = fvm.gradient_edges(fd, nlev)
            d = fvm.divergence_edges(ud, vd, nlev)
            lap = fvm.laplacian_edges(fd, nlev)
            torch.cuda.synchronize()
            for a, b in ((gx, om.gradient(f, nlev)[0]), (gy, om.gradient(f, nlev)[1]),
                         (d, om.divergence(u, v, nlev)), (lap, om.laplacian(f, nlev))):
                e = relmax(a[:, :nlev].double().cpu().numpy(), b)
                assert e <= tol[name], (N, name, "edges", e)
                worst[name] = max(worst[name], e)
                cases += 1
            # band partitions: halo windows shifted to global node ids
            for op in ("gradient", "laplacian", "divergence"):
                want = oracle_op(om, op, u if op in TWO_IN else f, v, nlev)
                full = (ud, vd) if op in TWO_IN else (fd,)
                for p in range(2):
                    part = partition.Partition(fvm, 2, p, 2 if op == "laplacian" else 1)
                    ins = [t[part.halo0:part.halo1].contiguous() for t in full]
                    outs = [torch.zeros((part.own1 - part.own0, ld), dtype=dt, device="cuda") for _ in want]
                    part.apply(op, ins, outs, nlev)
                    torch.cuda.synchronize()
                    for a, b in zip(outs, want):
                        e = relmax(a[:, :nlev].double().cpu().numpy(), b[part.own0:part.own1])
                        assert e <= tol[name], (N, name, "partition", op, p, e)
                        worst[name] = max(worst[name], e)
                        cases += 1
                    part.close()
            # a batched launch over both operators of the batch kernel
            jobs = [dict(op="gradient", fvm=fvm, ins=(fd,), outs=(torch.zeros_like(fd), torch.zeros_like(fd)),
                         nlev=nlev, N=N),
                    dict(op="divergence", fvm=fvm, ins=(ud, vd), outs=(torch.zeros_like(fd),), nlev=nlev, N=N)]
            b = batch.Batch(jobs)
            b.launch()
            torch.cuda.synchronize()
            for a, w in zip(jobs[0]["outs"] + jobs[1]["outs"], om.gradient(f, nlev) + (om.divergence(u, v, nlev),)):
                e = relmax(a[:, :nlev].double().cpu().numpy(), w)
                assert e <= tol[name], (N, name, "batch", e)
                worst[name] = max(worst[name], e)
                cases += 1
            b.close()
        # remap to the regular Gaussian grid F1 (its rows lie between the source rows)
        r = atlas.Remap(fvm.mesh, atlas.Grid(1, regular=True))
        a = r.grid.arrays()
        tgt = np.stack([a["lon"], a["lat_node"]], 1)
        f = synthetic.level_scalar(lon, lat, 5)
        out = r.apply(torch.from_numpy(synthetic.padded(f, 6)).cuda(), 5)
        torch.cuda.synchronize()
        e = relmax(out[:, :5].cpu().numpy(), om.remap(tgt, f, 5))
        assert e <= 1e-13, ("remap", e)
        worst["f64"] = max(worst["f64"], e)
        cases += 1
    status = atlas.kernel_status()
    print(json.dumps({"info": atlas.capi.atlas_info().decode(), "cases": cases, "worst": worst, "status": status}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
