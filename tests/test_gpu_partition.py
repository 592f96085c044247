"""GPU: band partitions and level shards give the whole-grid results bitwise.

The parts are emulated on one GPU, one after the other: each part's local
input is the whole field's halo range (what the halo exchange delivers),
``atlas_part_apply`` computes its own nodes, and the assembled outputs must
equal the whole-grid operator's, bit for bit (same kernels, same summation
order, only the node range and the buffers differ).  Level shards are column
views of the whole fields passed to the whole-grid calls."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


OPS = [("gradient", 1, 2), ("divergence", 2, 1), ("laplacian", 1, 1), ("gradient_adjoint", 2, 1),
       ("divergence_adjoint", 1, 2), ("curl", 2, 1), ("vector_gradient", 1, 2)]


def _whole(fvm, op, ins, nlev):
    if op == "gradient":
        return list(fvm.gradient(ins[0], nlev))
    if op == "divergence":
        return [fvm.divergence(ins[0], ins[1], nlev)]
    if op == "laplacian":
        return [fvm.laplacian(ins[0], nlev)]
    if op == "gradient_adjoint":
        return [fvm.gradient_adjoint(ins[0], ins[1], nlev)]
    if op == "divergence_adjoint":
        return list(fvm.divergence_adjoint(ins[0], nlev))
    if op == "curl":
        return [fvm.curl(ins[0], ins[1], nlev)]
    # one component through the vector-gradient table: compare with the
    # whole-grid call's first component
    return list(fvm.vector_gradient(ins[0], ins[0].clone(), nlev)[:2])


@pytest.mark.parametrize("dtype,ld", [("float32", 140), ("float64", 138), ("bfloat16", 144)])
def test_partitions_equal_whole_grid(torch, pfvm, dtype, ld):
    from paper_1908_07038_gb300.partition import Partition
    dt = getattr(torch, dtype)
    fvm = pfvm(80)
    nlev = 137
    gen = torch.Generator(device="cuda").manual_seed(2)
    fields = [torch.randn((fvm.nnodes, ld), generator=gen, device="cuda").to(dt) for _ in range(2)]
    for op, nin, nout in OPS:
        ins = fields[:nin]
        want = _whole(fvm, op, ins, nlev)
        halo = 2 if op == "laplacian" else 1
        for nparts in (2, 3, 5):
            got = [torch.full_like(want[0], float("nan")) for _ in range(nout)]
            for k in range(nparts):
                p = Partition(fvm, nparts, k, halo)
                local = [p.local_view(x).clone() for x in ins]
                outs = [torch.empty((p.own_rows, ld), dtype=dt, device="cuda") for _ in range(nout)]
                p.apply(op, local, outs, nlev)
                for g_, o in zip(got, outs):
                    g_[p.own0:p.own1] = o
                p.close()
            torch.cuda.synchronize()
            for g_, w in zip(got, want):
                assert torch.equal(g_[:, :nlev], w[:, :nlev]), (op, nparts, dtype)


def test_partition_rejects_wrong_shapes(torch, pfvm):
    from paper_1908_07038_gb300.partition import Partition
    from paper_1908_07038_gb300.capi import AtlasError
    fvm = pfvm(16)
    p = Partition(fvm, 2, 0, 1)
    f = torch.zeros((p.local_rows, 8), device="cuda")
    with pytest.raises(ValueError):
        p.apply("gradient", [f[:-1]], [torch.zeros((p.own_rows, 8), device="cuda")] * 2)
    with pytest.raises(AtlasError):  # the Laplacian needs a two-row halo
        p.apply("laplacian", [f], [torch.zeros((p.own_rows, 8), device="cuda")])
    p.close()


@pytest.mark.parametrize("nparts", [2, 3, 8])
def test_level_shards_equal_whole_levels(torch, pfvm, nparts):
    from paper_1908_07038_gb300.partition import level_shards
    fvm = pfvm(80)
    gen = torch.Generator(device="cuda").manual_seed(3)
    f, u, v = (torch.randn((fvm.nnodes, 140), generator=gen, device="cuda") for _ in range(3))
    gx, gy = fvm.gradient(f, 137)
    d = fvm.divergence(u, v, 137)
    lap = fvm.laplacian(f, 137)
    for a, b in level_shards(137, nparts):
        if a == b:
            continue
        sx = torch.zeros_like(f)
        sy = torch.zeros_like(f)
        sd = torch.zeros_like(f)
        sl = torch.zeros_like(f)
        fvm.gradient(f[:, a:], b - a, out=(sx[:, a:], sy[:, a:]))
        fvm.divergence(u[:, a:], v[:, a:], b - a, out=sd[:, a:])
        fvm.laplacian(f[:, a:], b - a, out=sl[:, a:])
        torch.cuda.synchronize()
        for s_, w in ((sx, gx), (sy, gy), (sd, d), (sl, lap)):
            assert torch.equal(s_[:, a:b], w[:, a:b]), (a, b)


@pytest.mark.parametrize("dtype,ld", [("float32", 140), ("float64", 138)])
def test_interior_then_boundary_equals_whole_grid(torch, pfvm, dtype, ld):
    """The overlapped schedule on one GPU: each part computes its interior
    nodes (no halo needed) and then the rows next to its halo, with
    ``apply_nodes``; the assembled outputs equal the whole-grid operators
    bitwise."""
    from paper_1908_07038_gb300.partition import Partition
    dt = getattr(torch, dtype)
    fvm = pfvm(80)
    nlev = 137
    gen = torch.Generator(device="cuda").manual_seed(4)
    fields = [torch.randn((fvm.nnodes, ld), generator=gen, device="cuda").to(dt) for _ in range(2)]
    for op, nin, nout in OPS[:6]:
        ins = fields[:nin]
        want = _whole(fvm, op, ins, nlev)
        halo = 2 if op == "laplacian" else 1
        got = [torch.full_like(want[0], float("nan")) for _ in range(nout)]
        for k in range(3):
            p = Partition(fvm, 3, k, halo)
            local = [p.local_view(x).clone() for x in ins]
            outs = [torch.full((p.own_rows, ld), float("nan"), dtype=dt, device="cuda") for _ in range(nout)]
            i0, i1 = p.interior
            assert p.own0 <= i0 < i1 <= p.own1
            p.apply_nodes(op, local, outs, i0, i1 - i0, nlev)
            p.apply_nodes(op, local, outs, p.own0, i0 - p.own0, nlev)
            p.apply_nodes(op, local, outs, i1, p.own1 - i1, nlev)
            for g_, o in zip(got, outs):
                g_[p.own0:p.own1] = o
            p.close()
        torch.cuda.synchronize()
        for g_, w in zip(got, want):
            assert torch.equal(g_[:, :nlev], w[:, :nlev]), (op, dtype)


# --------------------------------------------------- against the FP64 oracle
ORACLE_OPS = [("gradient", 1, 2), ("divergence", 2, 1), ("laplacian", 1, 1), ("gradient_adjoint", 2, 1),
              ("divergence_adjoint", 1, 2), ("curl", 2, 1), ("curl_adjoint", 1, 2), ("vector_gradient", 1, 2)]


def _oracle(om, op, ins, nlev):
    if op == "gradient":
        return list(om.gradient(ins[0], nlev))
    if op == "divergence":
        return [om.divergence(ins[0], ins[1], nlev)]
    if op == "laplacian":
        return [om.laplacian(ins[0], nlev)]
    if op == "gradient_adjoint":
        return [om.gradient_adjoint(ins[0], ins[1], nlev)]
    if op == "divergence_adjoint":
        return list(om.divergence_adjoint(ins[0], nlev))
    if op == "curl":
        return [om.curl(ins[0], ins[1], nlev)]
    if op == "curl_adjoint":
        return list(om.curl_adjoint(ins[0], nlev))
    return list(om.vector_gradient(ins[0], ins[0], nlev)[:2])  # the partition applies one component's table


@pytest.mark.parametrize("dtype,ld,tol", [("float32", 140, 1e-5), ("float64", 138, 1e-13)])
@pytest.mark.parametrize("overlapped", [False, True])
def test_partitions_against_oracle(torch, pfvm, omesh, dtype, ld, tol, overlapped):
    """Every operator on 3 band partitions of O80 x 137 (plain, or the
    overlapped interior-then-boundary schedule), assembled, against the FP64
    oracle on the same inputs (the recipe's fields, rounded to the dtype)."""
    import numpy as np
    import synthetic
    from paper_1908_07038_gb300.partition import Partition
    dt = getattr(torch, dtype)
    np_dt = np.float32 if dtype == "float32" else np.float64
    fvm, om = pfvm(80), omesh(80)
    g = om.grid()
    nlev = 137
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, np_dt)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, np_dt)
    dev = lambda x: torch.from_numpy(synthetic.padded(x, ld)).cuda()
    fields = {1: [dev(f)], 2: [dev(u), dev(v)]}
    host = {1: [f], 2: [u, v]}
    for op, nin, nout in ORACLE_OPS:
        ins = fields[nin]
        halo = 2 if op == "laplacian" else 1
        got = [torch.full((fvm.nnodes, ld), float("nan"), dtype=dt, device="cuda") for _ in range(nout)]
        for k in range(3):
            p = Partition(fvm, 3, k, halo)
            local = [p.local_view(x).clone() for x in ins]
            outs = [torch.empty((p.own_rows, ld), dtype=dt, device="cuda") for _ in range(nout)]
            if overlapped:
                i0, i1 = p.interior
                p.apply_nodes(op, local, outs, i0, i1 - i0, nlev)
                p.apply_nodes(op, local, outs, p.own0, i0 - p.own0, nlev)
                p.apply_nodes(op, local, outs, i1, p.own1 - i1, nlev)
            else:
                p.apply(op, local, outs, nlev)
            for g_, o in zip(got, outs):
                g_[p.own0:p.own1] = o
            p.close()
        torch.cuda.synchronize()
        want = _oracle(om, op, host[nin], nlev)
        for c, (g_, w) in enumerate(zip(got, want)):
            a = g_[:, :nlev].double().cpu().numpy()
            err = np.max(np.abs(a - w)) / np.max(np.abs(w))
            assert err <= tol, (op, c, dtype, overlapped, err)


@pytest.mark.parametrize("dtype,ld,tol", [("float32", 140, 1e-5), ("float64", 138, 1e-13)])
def test_level_shards_against_oracle(torch, pfvm, omesh, dtype, ld, tol):
    """The seven whole-grid operators applied to three level shards of O80 x
    137 (column views starting on 16-byte boundaries), assembled, against
    the FP64 oracle on the same inputs."""
    import numpy as np
    import synthetic
    from paper_1908_07038_gb300.partition import level_shards
    dt = getattr(torch, dtype)
    np_dt = np.float32 if dtype == "float32" else np.float64
    fvm, om = pfvm(80), omesh(80)
    g = om.grid()
    nlev = 137
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev, np_dt)
    u, v = synthetic.level_vector(g["lon"], g["lat_node"], nlev, np_dt)
    dev = lambda x: torch.from_numpy(synthetic.padded(x, ld)).cuda()
    fields = {1: [dev(f)], 2: [dev(u), dev(v)]}
    host = {1: [f], 2: [u, v]}
    calls = {"gradient": lambda i, n, o: fvm.gradient(i[0], n, out=tuple(o)),
             "divergence": lambda i, n, o: fvm.divergence(i[0], i[1], n, out=o[0]),
             "laplacian": lambda i, n, o: fvm.laplacian(i[0], n, out=o[0]),
             "gradient_adjoint": lambda i, n, o: fvm.gradient_adjoint(i[0], i[1], n, out=o[0]),
             "divergence_adjoint": lambda i, n, o: fvm.divergence_adjoint(i[0], n, out=tuple(o)),
             "curl": lambda i, n, o: fvm.curl(i[0], i[1], n, out=o[0]),
             "curl_adjoint": lambda i, n, o: fvm.curl_adjoint(i[0], n, out=tuple(o)),
             "vector_gradient": None}
    for op, nin, nout in ORACLE_OPS:
        if calls[op] is None:
            continue
        ins = fields[nin]
        got = [torch.full((fvm.nnodes, ld), float("nan"), dtype=dt, device="cuda") for _ in range(nout)]
        for a, b in level_shards(nlev, 3):
            if a == b:
                continue
            calls[op]([x[:, a:] for x in ins], b - a, [o[:, a:] for o in got])
        torch.cuda.synchronize()
        want = _oracle(om, op, host[nin], nlev)
        for c, (g_, w) in enumerate(zip(got, want)):
            a_ = g_[:, :nlev].double().cpu().numpy()
            err = np.max(np.abs(a_ - w)) / np.max(np.abs(w))
            assert err <= tol, (op, c, dtype, err)


def _nccl_rank(rank, port, out):
    """One rank of a one-process NCCL world: the partition calls that talk
    to torch.distributed run on CUDA tensors through the NCCL backend."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1908_07038_gb300 import atlas
    from paper_1908_07038_gb300.partition import Partition
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        fvm = atlas.build_fvm(32)
        gen = torch.Generator(device="cuda").manual_seed(6)
        x = torch.randn((fvm.nnodes, 12), generator=gen, device="cuda")
        u, v = fvm.gradient(x, 12)
        d = fvm.divergence(u, v, 12)
        p = Partition(fvm, 1, 0, 1)  # the whole grid as the one part: no neighbours
        local = p.local_view(u).clone()
        p.exchange(local)  # nothing to send: returns at once
        outs = [torch.empty((p.own_rows, 12), device="cuda")]
        p.apply_overlapped("divergence", [p.local_view(u).clone(), p.local_view(v).clone()], outs, 12)
        s = p.integral(outs[0], 12)  # all_reduce over NCCL
        w = fvm.integral(d, 12)
        torch.cuda.synchronize()
        ok = torch.equal(outs[0], d) and torch.equal(s, w)
        np.save(out, np.array([1.0 if ok else 0.0]))
        p.close()
    finally:
        dist.destroy_process_group()


def test_partition_calls_over_nccl_one_rank(torch, tmp_path):
    """The NCCL branch of the partition's collectives on CUDA tensors, in a
    world of one rank (exchange with no neighbours, the overlapped schedule,
    the all-reduce of the conservation sums).  Exchanges between ranks need
    two GPUs and are tested over gloo on CPU instead."""
    import socket
    import numpy as np
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "nccl_ok.npy")
    mp.spawn(_nccl_rank, args=(port, out), nprocs=1, join=True)
    assert np.load(out)[0] == 1.0
