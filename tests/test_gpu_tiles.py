"""GPU: the shared-memory node-group (tile) kernels against the per-node
kernels, bit for bit, and their bounded waits.

The tile kernels accumulate every node's terms in the per-node kernels'
order with the same operations, so the two give identical bits; the
per-node kernels are themselves pinned to the FP64 oracle by the parity
tests.  Covered: every operator, FP32 and BF16 storage, tiles of 1, 3 and
7 groups, ragged level counts (every part A / part B
level layout), O, F and regional grids, and whole-row node ranges
(partitions).  The time-out path of the pipeline waits is run with the
testing hook that makes the consumers wait on a barrier nothing completes:
the kernel returns, the status word says so, and the next launches are
correct again (no GPU fault, no hang).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OPS = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint", "curl", "vector_gradient",
       "curl_adjoint")
NIN = {"divergence": 2, "gradient_adjoint": 2, "curl": 2, "vector_gradient": 2}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


NOUT = {"gradient": 2, "divergence_adjoint": 2, "vector_gradient": 4, "curl_adjoint": 2}
# the library's default groups per tile, per operator and storage (F32, F64, BF16)
DEFAULT_GROUPS = {op: (12, 7, 15) if op == "laplacian" else
                  (10, 7, 15) if op in ("gradient", "divergence_adjoint", "vector_gradient", "curl_adjoint") else
                  (10, 7, 11) for op in OPS}
DEFAULT_ROWS = {op: (2, 1, 1) for op in OPS}


def _call(fvm, op, x, y, nlev, out=None):
    """One operator; out: preallocated outputs (else fresh ones)."""
    if out is None:
        out = [fvm._out(x, None) for _ in range(NOUT.get(op, 1))]
    if op == "gradient":
        return fvm.gradient(x, nlev, out=tuple(out))
    if op == "divergence":
        return (fvm.divergence(x, y, nlev, out=out[0]),)
    if op == "laplacian":
        return (fvm.laplacian(x, nlev, out=out[0]),)
    if op == "gradient_adjoint":
        return (fvm.gradient_adjoint(x, y, nlev, out=out[0]),)
    if op == "divergence_adjoint":
        return fvm.divergence_adjoint(x, nlev, out=tuple(out))
    if op == "curl":
        return (fvm.curl(x, y, nlev, out=out[0]),)
    if op == "vector_gradient":
        return fvm.vector_gradient(x, y, nlev, out=tuple(out))
    return fvm.curl_adjoint(x, nlev, out=tuple(out))


def _filled(torch, x, n):
    return [torch.full_like(x, 7.0) for _ in range(n)]


def _compare(torch, fvm, x, y, nlev, groups=(11, 7, 3, 1), ops=OPS, npws=(4, 2)):
    """Every operator with the tile kernels (tiles of several sizes, one or
    two consumer warps per group; with one warp per group, the tables with
    union groups and without) against the per-node kernels: identical
    outputs, padding included (outputs start filled with 7: the levels past
    the stored vectors must keep it).  Shapes the kernels cannot take (two
    warps per group in tiles of eleven groups, stages too large) run per
    node and compare trivially."""
    from paper_1908_07038_gb300 import capi
    dt = {torch.float32: 0, torch.float64: 1, torch.bfloat16: 2}[x.dtype]
    shapes = [(w, u, 1) for w in npws for u in ((1, 0) if w == 4 else (1,))]
    if 4 in npws:
        shapes += [(4, 1, 2), (4, 0, 2), (4, 1, 3)]  # tiles spanning two and three grid rows
    for op in ops:
        n = NOUT.get(op, 1)
        fvm.set_group(op, enable=0, dtype=dt)
        ref = _call(fvm, op, x, y, nlev, _filled(torch, x, n))
        for gpt in groups:
            for npw, unions, rows in shapes:
                capi.atlas_debug_tile_unions(unions)
                try:
                    fvm.set_group(op, enable=2, groups_per_tile=gpt, nodes_per_warp=npw, dtype=dt, rows_per_tile=rows)
                    got = _call(fvm, op, x, y, nlev, _filled(torch, x, n))
                    torch.cuda.synchronize()
                finally:
                    capi.atlas_debug_tile_unions(1)
                for a, b in zip(got, ref):
                    assert torch.equal(a, b), (op, gpt, npw, unions, rows)
        fvm.set_group(op, enable=1, groups_per_tile=DEFAULT_GROUPS[op][dt], nodes_per_warp=4, dtype=dt,
                      rows_per_tile=DEFAULT_ROWS[op][dt])


def _fields(torch, V, ld, dt, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return [torch.randn((V, ld), device="cuda", generator=g).to(dt) for _ in range(2)]


@pytest.mark.parametrize("nlev,ld", [(137, 140), (137, 160), (1, 4), (30, 32), (60, 64), (91, 92), (128, 128),
                                     (150, 152), (200, 200), (300, 300)])
def test_tiles_equal_per_node_kernels_fp32(torch, pfvm, nlev, ld):
    """All level layouts (va, vb): 1 level, 32, 64, 96, 128, 160, 192 and
    several level blocks."""
    fvm = pfvm(16)
    x, y = _fields(torch, fvm.nnodes, ld, torch.float32, nlev)
    _compare(torch, fvm, x, y, nlev)


def test_tiles_equal_per_node_kernels_bf16(torch, pfvm):
    fvm = pfvm(32)
    for nlev, ld in ((137, 144), (9, 16), (64, 64)):
        x, y = _fields(torch, fvm.nnodes, ld, torch.bfloat16, nlev)
        _compare(torch, fvm, x, y, nlev)


def test_tiles_on_f_and_regional_grids(torch, product):
    atlas, _ = product
    from synthetic.regional import DOMAINS
    grids = [atlas.build_fvm(24, regular=True)]
    for name in ("lambert", "rotated", "polar"):
        proj, kw = DOMAINS[name]
        grids.append(atlas.build_fvm_regional(proj, 37, 23, **kw))  # 37 per row: rows of 9 groups and a short one
    for fvm in grids:
        x, y = _fields(torch, fvm.nnodes, 140, torch.float32, 3)
        _compare(torch, fvm, x, y, 137, groups=(7, 2))
        # away from their edges these grids have the octahedral interior's
        # neighbourhood: the default tables hold union groups for them too
        for op in ("gradient", "divergence", "laplacian"):
            assert fvm.tile_union_groups(op) > 0, op


def test_tiles_o1280_benchmark_layout(torch, pfvm):
    """The benchmark workload's grid and layout (O1280 x 137, ld 140): the
    default tile kernels against the per-node kernels for every operator."""
    fvm = pfvm(1280)
    x, y = _fields(torch, fvm.nnodes, 140, torch.float32, 11)
    _compare(torch, fvm, x, y, 137, groups=(7,))
    # with one warp per group almost every group takes the union form
    for op in OPS:
        ng = sum(-(-p // 4) for p in fvm.grid.arrays()["pl"])
        assert fvm.tile_union_groups(op) > 0.95 * ng, op
    del x, y
    torch.cuda.empty_cache()


def test_tiles_in_partitions(torch, pfvm):
    """Band partitions launch the tile kernels on whole rows of their own
    nodes (halo buffers shifted to global node ids): identical to the
    whole-grid result."""
    from paper_1908_07038_gb300 import partition
    fvm = pfvm(32)
    x, y = _fields(torch, fvm.nnodes, 140, torch.float32, 5)
    for op in ("gradient", "divergence", "laplacian", "curl_adjoint"):
        whole = [t.clone() for t in _call(fvm, op, x, y, 137)]
        for nparts in (2, 3):
            rings = 2 if op == "laplacian" else 1
            for p in range(nparts):
                part = partition.Partition(fvm, nparts, p, rings)
                h0, h1, o0, o1 = part.halo0, part.halo1, part.own0, part.own1
                ins = [x[h0:h1].contiguous()] + ([y[h0:h1].contiguous()] if NIN.get(op, 1) == 2 else [])
                outs = [torch.full((o1 - o0, 140), 7.0, device="cuda") for _ in whole]
                part.apply(op, ins, outs, 137)
                torch.cuda.synchronize()
                for a, b in zip(outs, whole):
                    assert torch.equal(a, b[o0:o1]), (op, nparts, p)
                part.close()


def test_bounded_wait_reports_and_recovers(torch, product, pfvm):
    """The consumers wait on a barrier nothing completes: past a limit of a
    few milliseconds the kernel records code 1 (and the producer, whose
    stages are never released, code 2) and returns; afterwards the status
    clears and the operators are correct again."""
    atlas, capi = product
    fvm = pfvm(16)
    x, y = _fields(torch, fvm.nnodes, 140, torch.float32, 9)
    fvm.set_group("gradient", enable=0)
    ref = [t.clone() for t in fvm.gradient(x, 137)]
    fvm.set_group("gradient", enable=1)
    assert atlas.kernel_status() == 0
    capi.atlas_debug_tile_hang(1)
    try:
        fvm.gradient(x, 137)
        code = atlas.kernel_status()
    finally:
        capi.atlas_debug_tile_hang(0)
    assert code & 1, code
    assert atlas.kernel_status() == 0  # cleared by the read above
    got = fvm.gradient(x, 137)
    torch.cuda.synchronize()
    assert atlas.kernel_status() == 0
    assert torch.equal(got[0][:, :140], ref[0][:, :140]) and torch.equal(got[1][:, :140], ref[1][:, :140])
