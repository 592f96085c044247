"""Host-side logic of the multi-rank benchmark, on CPU with the gloo backend.

The operators need no exchange, so under torchrun every rank runs an
independent replica; what the ranks share is the timing rule (the job takes
as long as its slowest rank) and the throughput rule (all ranks' units over
that time), and only rank 0 prints.  Two ranks run here as processes on CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        # rank r "took" 10 + 5 r ms; every rank must see the slowest
        slowest = bench._max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        rate = bench._job_rate(1000, world, slowest)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
            fh.write("%r %r\n" % (slowest, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        slowest, rate = (float(x) for x in (tmp_path / ("rank%d.txt" % r)).read_text().split())
        assert slowest == 15.0
        assert rate == pytest.approx(world * 1000 / 15e-3, rel=1e-15)
    del torch


def test_single_rank_needs_no_process_group():
    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench._job_rate(10, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle arm runs on rank 0; other ranks return at once
    without work or output."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(None) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle timed on host cores over a
    bounded node sample) prints exactly one JSON line with the keys the
    benchmark contract fixes, its e2e and cpu_baseline describing the same run."""
    import json
    import subprocess
    env = dict(os.environ, ORACLE_STEP_SECONDS="0.2", WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [s for s in out.stdout.splitlines() if s.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["unit"] == line["e2e"]["unit"] == line["cpu_baseline"]["unit"]
    assert line["e2e"]["value"] == line["value"] == line["cpu_baseline"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "workload" in line["config"] and line["cpu_baseline"]["sample"]


def test_algorithmic_table_bytes_follow_the_mesh_counts(pfvm):
    """The roofline's table bytes: offsets, then 12 bytes per entry (index +
    two FP32 weights) or 8 (the Laplacian's one weight), plus 8 bytes per
    node for a B term.  The entry counts come from the mesh: 2E for the
    gradient and its adjoint (every edge seen from both ends), 2E - 2P for
    the divergence and its adjoint (P pole edges carry no flux), and for the
    Laplacian L = D G the nodes that G reaches from the node itself or from
    a neighbour across a face that carries divergence flux (so not across a
    pole edge), the node itself excluded."""
    fvm = pfvm(16)
    V, E = fvm.nnodes, fvm.mesh.nedges
    m = fvm.mesh.arrays()
    P = int(m["is_pole"].sum())
    assert E == 3 * V - 20 and P == 20
    offsets = 4 * (V + 1)
    want = {"gradient": offsets + 2 * E * 12,
            "gradient_adjoint": offsets + 2 * E * 12 + 8 * V,
            "divergence": offsets + (2 * E - 2 * P) * 12 + 8 * V,
            "divergence_adjoint": offsets + (2 * E - 2 * P) * 12 + 8 * V}
    for op, b in want.items():
        assert bench._table_bytes_of(fvm, op, 4) == b, op
    # the Laplacian's neighbourhoods by brute force over the edge list
    nb = [set() for _ in range(V)]  # gradient neighbours (every edge)
    nd = [set() for _ in range(V)]  # divergence neighbours (no pole edges)
    for (a, c), pole in zip(m["e2n"], m["is_pole"]):
        nb[a].add(c)
        nb[c].add(a)
        if not pole:
            nd[a].add(c)
            nd[c].add(a)
    ring2 = sum(len(set().union(nb[i], *(nb[j] for j in nd[i])) - {i}) for i in range(V))
    assert bench._table_bytes_of(fvm, "laplacian", 4) == offsets + ring2 * 8


def test_traffic_only_for_the_kernels_it_was_measured_on(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu capture only while the
    kernel source hashes to the value stored with it; otherwise it is null."""
    import hashlib
    import json
    src = tmp_path / "kernels.cu"
    src.write_text("// kernels, version 1\n")
    cap = tmp_path / "traffic.json"
    good = hashlib.sha256(src.read_bytes()).hexdigest()
    cap.write_text(json.dumps({"kernels_sha256": good, "per_launch_bytes": {"gradient": 123.0}}))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", (str(src),))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(cap))
    assert bench._traffic("gradient") == 123.0
    assert bench._traffic("laplacian") is None  # not captured
    src.write_text("// kernels, version 2\n")
    assert bench._traffic("gradient") is None  # the kernels changed since
    cap.unlink()
    assert bench._traffic("gradient") is None
    # the committed capture matches the committed kernels (after a kernel
    # change, take the capture again: profiles/dram_traffic_o1280.json)
    monkeypatch.undo()
    for op in ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint"):
        assert bench._traffic(op) is not None, "no DRAM traffic for %s: the kernel sources changed since the capture" % op


def test_peak_is_the_measured_copy_rate_else_the_fallback(tmp_path, monkeypatch):
    import json
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6768.8, "bf16_tflops": 1900}))
    assert bench._peaks() == (6768.8, "measured")
