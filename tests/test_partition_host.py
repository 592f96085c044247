"""Band partitions (host side) and the halo exchange, on CPU.

The partition geometry comes from the C ABI without a GPU; the exchange runs
as gloo ranks on CPU tensors.  What is checked: the parts tile the nodes
with whole rows, every stencil neighbour of an own node lies in the part's
halo range (one ring, or two for the fused Laplacian), the send and receive
ranges of adjacent parts match, and after one exchange every part's local
field equals the whole field on its halo range."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def part_mod(product):
    from paper_1908_07038_gb300 import partition
    return partition


@pytest.mark.parametrize("halo", [1, 2])
@pytest.mark.parametrize("nparts", [1, 2, 3, 5, 8])
def test_parts_tile_the_nodes_in_whole_rows(pfvm, part_mod, nparts, halo):
    fvm = pfvm(16)
    off = np.concatenate([[0], np.cumsum(fvm.grid.arrays()["pl"])])
    parts = [part_mod.Partition(fvm, nparts, p, halo) for p in range(nparts)]
    assert parts[0].own0 == 0 and parts[-1].own1 == fvm.nnodes
    for a, b in zip(parts, parts[1:]):
        assert a.own1 == b.own0
    sizes = []
    for p in parts:
        r0, r1 = np.searchsorted(off, p.own0), np.searchsorted(off, p.own1)
        assert off[r0] == p.own0 and off[r1] == p.own1 and r1 - r0 >= halo
        assert p.halo0 == off[max(0, r0 - halo)] and p.halo1 == off[min(len(off) - 1, r1 + halo)]
        sizes.append(p.own1 - p.own0)
    # about equal shares: no part more than one row's worth off the mean
    assert max(sizes) - min(sizes) <= 2 * max(np.diff(off)) + 1
    for p in parts:
        p.close()


@pytest.mark.parametrize("op,halo", [("gradient", 1), ("divergence", 1), ("curl", 1), ("gradient_adjoint", 1),
                                     ("divergence_adjoint", 1), ("vector_gradient", 1), ("laplacian", 2)])
def test_halo_holds_every_stencil_neighbour(pfvm, part_mod, op, halo):
    fvm = pfvm(16)
    t = fvm.stencil_table(op)
    ptr, nbr = t["ptr"], t["nbr"]
    for nparts in (2, 4, 7):
        for k in range(nparts):
            p = part_mod.Partition(fvm, nparts, k, halo)
            cols = nbr[ptr[p.own0]:ptr[p.own1]]
            assert cols.min() >= p.halo0 and cols.max() < p.halo1
            p.close()


@pytest.mark.parametrize("family", ["F16", "lambert", "polar", "rotated"])
def test_bands_and_halos_on_other_grid_families(product, part_mod, family):
    """The regular Gaussian grid and regional grids (rows of a projection's
    plane) partition the same way: whole rows, and every stencil neighbour
    of every operator within the one-row halo (two rows for the Laplacian)."""
    atlas, _ = product
    from synthetic.regional import DOMAINS
    if family == "F16":
        fvm = atlas.build_fvm(16, regular=True)
        rows = np.full(32, 64)
    else:
        proj, kw = DOMAINS[family]
        fvm = atlas.build_fvm_regional(proj, 23, 19, **kw)
        rows = np.full(19, 23)
    off = np.concatenate([[0], np.cumsum(rows)])
    for op in ("gradient", "divergence", "curl", "gradient_adjoint", "divergence_adjoint", "vector_gradient",
               "laplacian"):
        halo = 2 if op == "laplacian" else 1
        t = fvm.stencil_table(op)
        for nparts in (2, 3, 6):
            parts = [part_mod.Partition(fvm, nparts, k, halo) for k in range(nparts)]
            assert parts[0].own0 == 0 and parts[-1].own1 == fvm.nnodes
            for a, b in zip(parts, parts[1:]):
                assert a.own1 == b.own0
            for p in parts:
                assert p.own0 in off and p.own1 in off and p.halo0 in off and p.halo1 in off
                cols = t["nbr"][t["ptr"][p.own0]:t["ptr"][p.own1]]
                assert cols.min() >= p.halo0 and cols.max() < p.halo1, (family, op, nparts)
                p.close()


def test_neighbour_ranges_match(pfvm, part_mod):
    fvm = pfvm(16)
    for halo in (1, 2):
        parts = [part_mod.Partition(fvm, 4, k, halo) for k in range(4)]
        for k, p in enumerate(parts):
            for n in p.neighbours:
                q = parts[n["peer"]]
                back = [m for m in q.neighbours if m["peer"] == k][0]
                assert back["recv"] == n["send"] and back["send"] == n["recv"]
                assert p.own0 <= n["send"][0] < n["send"][1] <= p.own1
                assert p.halo0 <= n["recv"][0] < n["recv"][1] <= p.halo1
                assert not (p.own0 <= n["recv"][0] < p.own1)
        for p in parts:
            p.close()


def test_partition_errors(pfvm, part_mod, product):
    atlas, capi = product
    fvm = pfvm(8)  # 16 rows
    with pytest.raises(capi.AtlasError):
        part_mod.Partition(fvm, 9, 0, 2)  # 9 parts of >= 2 rows do not fit 16 rows
    with pytest.raises(capi.AtlasError):
        part_mod.Partition(fvm, 2, 2, 1)
    with pytest.raises(capi.AtlasError):
        part_mod.Partition(fvm, 2, 0, 3)
    f2 = atlas.build_fvm(4)
    p = part_mod.Partition(f2, 2, 0, 1)
    f2.close()  # refused while the partition holds it: the handle stays valid
    assert p.own1 > 0
    p.close()


def test_level_shards(part_mod):
    for nlev, n in ((137, 2), (137, 3), (137, 8), (5, 4), (1, 1)):
        sh = part_mod.level_shards(nlev, n)
        assert sh[0][0] == 0 and sh[-1][1] == nlev and len(sh) == n
        for (_, b), (c, _) in zip(sh, sh[1:]):
            assert b == c
        for a, b in sh:
            assert a % 4 == 0 and a <= b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_rank(rank, world, port, halo, out_dir):
    import torch
    import torch.distributed as dist
    from paper_1908_07038_gb300 import atlas
    from paper_1908_07038_gb300.partition import Partition
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        fvm = atlas.build_fvm(16)
        whole = torch.from_numpy(np.random.default_rng(9).standard_normal((fvm.nnodes, 6)))
        p = Partition(fvm, world, rank, halo)
        local = torch.full((p.local_rows, 6), float("nan"), dtype=torch.float64)
        p.own_of_local(local).copy_(whole[p.own0:p.own1])
        p.exchange(local)
        ok = torch.equal(local, whole[p.halo0:p.halo1])
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
            fh.write("ok" if ok else "mismatch")
        p.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,halo", [(2, 1), (3, 2)])
def test_halo_exchange_gloo(tmp_path, product, world, halo):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(_exchange_rank, args=(world, _free_port(), halo, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        assert (tmp_path / ("rank%d.txt" % r)).read_text() == "ok"


def _integral_rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    from paper_1908_07038_gb300 import atlas
    from paper_1908_07038_gb300.partition import Partition
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        fvm = atlas.build_fvm(16)
        V = torch.from_numpy(fvm.arrays()["V"])

        # host stand-in for the device sum (the kernel needs a GPU): the same
        # contract, FP64 sums over the given node range
        def host_integral(x, nlev=None, node0=0, count=None, out=None, ws=None):
            count = x.shape[0] if count is None else count
            nlev = x.shape[1] if nlev is None else nlev
            return (V[node0:node0 + count, None] * x[:count, :nlev].double()).sum(0)

        fvm.integral = host_integral
        whole = torch.from_numpy(np.random.default_rng(10).standard_normal((fvm.nnodes, 5)))
        p = Partition(fvm, world, rank, 1)
        got = p.integral(whole[p.own0:p.own1])
        want = host_integral(whole)
        ok = bool(torch.allclose(got, want, rtol=1e-13, atol=1e-13 * float((V[:, None] * whole.abs()).sum())))
        with open(os.path.join(out_dir, "int%d.txt" % rank), "w") as fh:
            fh.write("ok" if ok else "mismatch %r %r" % (got.tolist(), want.tolist()))
        p.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_partition_integral_all_reduce_gloo(tmp_path, product):
    """The parts' own-node sums added by all_reduce over gloo ranks equal the
    whole-grid sum on every rank."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(_integral_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert (tmp_path / ("int%d.txt" % r)).read_text() == "ok"


@pytest.mark.parametrize("nparts,halo", [(2, 1), (3, 2), (5, 1), (7, 2)])
def test_interior_reads_no_halo(pfvm, part_mod, nparts, halo):
    """Every node of a part's interior has all its stencil neighbours among
    the part's own nodes, and the interior spans the own rows less the halo
    rows on each side that has a neighbour."""
    fvm = pfvm(32)
    ops = ["gradient", "divergence", "curl"] + (["laplacian"] if halo == 2 else [])
    tabs = {op: fvm.stencil_table(op) for op in ops}
    pl = fvm.grid.arrays()["pl"]
    off = np.concatenate([[0], np.cumsum(pl)])
    for k in range(nparts):
        p = part_mod.Partition(fvm, nparts, k, halo)
        i0, i1 = p.interior
        assert p.own0 <= i0 <= i1 <= p.own1
        r0 = int(np.searchsorted(off, p.own0))
        r1 = int(np.searchsorted(off, p.own1))
        want0 = off[r0 + halo] if k > 0 else p.own0
        want1 = off[r1 - halo] if k < nparts - 1 else p.own1
        assert (i0, i1) == (want0, max(want0, want1))
        for op, t in tabs.items():
            lo, hi = t["ptr"][i0], t["ptr"][i1]
            nb = t["nbr"][lo:hi]
            assert nb.size == 0 or (nb.min() >= p.own0 and nb.max() < p.own1), (op, k)
        p.close()


def _overlap_rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    from paper_1908_07038_gb300 import atlas
    from paper_1908_07038_gb300.partition import Partition
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        fvm = atlas.build_fvm(16)
        t = fvm.stencil_table("gradient")
        ptr, nbr, w = t["ptr"], t["nbr"], t["w"]

        # host stand-in for the device kernels (they need a GPU): the FP64
        # gradient table applied to the rows [node0, node0 + count)
        def host_apply_nodes(p, op, ins, outs, node0, count, nlev=None):
            x = ins[0].numpy()
            for i in range(node0, node0 + count):
                q = slice(ptr[i], ptr[i + 1])
                d = x[nbr[q] - p.halo0] - x[i - p.halo0]
                for c in range(2):
                    outs[c][i - p.own0] = torch.from_numpy(w[q, c] @ d)

        whole = torch.from_numpy(np.random.default_rng(13).standard_normal((fvm.nnodes, 3)))
        p = Partition(fvm, world, rank, 1)
        p.apply_nodes = lambda op, ins, outs, node0, count, nlev=None: host_apply_nodes(p, op, ins, outs, node0,
                                                                                        count, nlev)
        local = torch.full((p.local_rows, 3), float("nan"), dtype=torch.float64)
        p.own_of_local(local).copy_(whole[p.own0:p.own1])
        outs = [torch.full((p.own_rows, 3), float("nan"), dtype=torch.float64) for _ in range(2)]
        p.apply_overlapped("gradient", [local], outs)
        full = Partition(fvm, 1, 0, 1)
        ref = [torch.zeros((fvm.nnodes, 3), dtype=torch.float64) for _ in range(2)]
        host_apply_nodes(full, "gradient", [whole], ref, 0, fvm.nnodes)
        ok = all(torch.equal(o, r[p.own0:p.own1]) for o, r in zip(outs, ref))
        with open(os.path.join(out_dir, "ov%d.txt" % rank), "w") as fh:
            fh.write("ok" if ok else "mismatch")
        p.close()
        full.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_overlapped_exchange_and_apply_gloo(tmp_path, product):
    """apply_overlapped over 2 gloo ranks (the device apply replaced by a host
    stand-in): interior first, halo in flight, then the boundary rows; equal
    to the whole-grid result, with no NaN from an unreceived halo."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(_overlap_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert (tmp_path / ("ov%d.txt" % r)).read_text() == "ok"


def test_apply_nodes_range_errors(pfvm, part_mod, product):
    """apply_nodes refuses ranges outside the part's own nodes before it
    touches any pointer (host-side check, no GPU needed)."""
    capi = product[1]
    fvm = pfvm(16)
    p = part_mod.Partition(fvm, 3, 1, 1)
    fake = 0x100000
    for node0, count in [(p.own0 - 1, 5), (p.own1 - 2, 5), (p.own0, -1)]:
        with pytest.raises(capi.AtlasError) as ei:
            capi.atlas_part_apply_nodes(p.handle, capi.ATLAS_OP_GRADIENT, fake, None, fake, fake, node0, count,
                                        4, 4, capi.ATLAS_F32, None)
        assert ei.value.code == -1
    with pytest.raises(capi.AtlasError):  # the Laplacian needs two halo rows
        capi.atlas_part_apply_nodes(p.handle, capi.ATLAS_OP_LAPLACIAN, fake, None, fake, None, p.own0, 1,
                                    4, 4, capi.ATLAS_F32, None)
    p.close()
