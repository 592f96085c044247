"""Host checks of the node-group tables (no GPU).

The group table is the union of the stencil rows of each group of up to
four consecutive nodes (what a tile stages).  Every node must find there
exactly its own stencil row, with the same weights.  These tests check that
on every grid family and operator, against the per-node table of the same
fvm, plus the group layout the kernels rely on (whole-row groups of at most
four nodes, sorted entries, the run of the group's own nodes), and the
entry order of the stencil rows that every kernel sums in: the neighbours on
the node's own grid row at offsets -2, -1, +1, +2 (those present) first,
then the others by ascending id.
"""
import numpy as np
import pytest

OPS = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint", "curl", "vector_gradient")


def _fvms(atlas):
    from synthetic.regional import DOMAINS
    proj, kw = DOMAINS["lambert"]
    return {"O2": atlas.build_fvm(2), "O9": atlas.build_fvm(9), "F6": atlas.build_fvm(6, regular=True),
            "lambert13x9": atlas.build_fvm_regional(proj, 13, 9, **kw),
            "lambert7x5": atlas.build_fvm_regional(proj, 7, 5, **kw)}


@pytest.fixture(scope="module")
def fvms(product):
    atlas, _ = product
    return _fvms(atlas)


def _rows(fvm):
    g = fvm.grid.arrays()
    return np.concatenate([[0], np.cumsum(g["pl"])]).astype(np.int64)


@pytest.mark.parametrize("name", ["O2", "O9", "F6", "lambert13x9", "lambert7x5"])
@pytest.mark.parametrize("op", OPS)
def test_group_table_reproduces_every_node_row(fvms, name, op):
    fvm = fvms[name]
    st = fvm.stencil_table(op)
    gt = fvm.group_table(op)
    head, hdr, w = gt["head"], gt["hdr"], gt["w"]
    ptr, nbr, sw = st["ptr"], st["nbr"], st["w"]
    V = fvm.nnodes
    off = _rows(fvm)
    nw = 1 if op == "laplacian" else 2
    # groups: consecutive, whole rows, at most four nodes, entries contiguous
    firsts = head[:, 0].astype(np.int64)
    counts = (head[:, 3] >> 16) & 0xF
    assert firsts[0] == 0 and np.all(firsts[1:] == firsts[:-1] + counts[:-1]) and firsts[-1] + counts[-1] == V
    assert np.all((counts >= 1) & (counts <= 4))
    row_of = np.searchsorted(off, firsts, side="right") - 1
    assert np.all(firsts + counts <= off[row_of + 1])  # a group never crosses a row end
    assert head[0, 1] == 0 and np.all(head[1:, 1] == head[:-1, 2]) and head[-1, 2] == hdr.size
    j_all = (hdr & 0x0FFFFFFF).astype(np.int64)
    mask_all = hdr >> 28
    assert np.all(mask_all != 0)  # every entry serves some node of its group
    for g in range(head.shape[0]):
        f0, q0, q1 = int(firsts[g]), int(head[g, 1]), int(head[g, 2])
        cnt, nb, imask = int(counts[g]), int(head[g, 3] & 0xFFFF), int((head[g, 3] >> 20) & 0xF)
        js, ms = j_all[q0:q1], mask_all[q0:q1]
        assert np.all(np.diff(js) > 0)  # ascending, distinct
        assert nb == int(np.sum(js < f0))
        own = js[(js >= f0) & (js < f0 + cnt)]
        assert imask == sum(1 << int(x - f0) for x in own)
        assert np.all(ms < (1 << cnt))  # no bit for a node past the group's end
        for t in range(cnt):
            i = f0 + t
            sel = (ms >> t) & 1 == 1
            order = np.argsort(nbr[ptr[i]:ptr[i + 1]], kind="stable")
            assert np.array_equal(js[sel], nbr[ptr[i]:ptr[i + 1]][order]), (name, op, i)
            assert np.array_equal(w[q0:q1][sel, t, :nw], sw[ptr[i]:ptr[i + 1], :nw][order]), (name, op, i)
            assert np.all(w[q0:q1][~sel, t] == 0.0)


@pytest.mark.parametrize("name", ["O2", "O9", "F6", "lambert13x9", "lambert7x5"])
@pytest.mark.parametrize("op", OPS)
def test_stencil_rows_put_row_neighbours_first(fvms, name, op):
    """Each row starts with the node's neighbours on its own grid row at
    offsets -2, -1, +1, +2 along the row (a ring on global grids), in that
    order, then lists the others by ascending id; on global grids every node
    of a row of more than four points has its -1 and +1 neighbours there
    (and the Laplacian its -2 and +2 ones too)."""
    fvm = fvms[name]
    st = fvm.stencil_table(op)
    ptr, nbr = st["ptr"], st["nbr"]
    off = _rows(fvm)
    ring = fvm.grid.projection is None
    for r in range(len(off) - 1):
        a, n = int(off[r]), int(off[r + 1] - off[r])
        for i in range(a, a + n):
            row = [int(j) for j in nbr[ptr[i]:ptr[i + 1]]]
            offs = []
            for j in row:
                if a <= j < a + n:
                    d = j - i
                    if ring:
                        d = (j - i) % n
                        if 2 * d > n:
                            d -= n
                    offs.append(d if d != 0 and abs(d) <= 2 else None)
                else:
                    offs.append(None)
            k = 0
            while k < len(row) and offs[k] is not None:
                k += 1
            head, rest = offs[:k], row[k:]
            assert head == sorted(head), (name, op, i, row)
            assert all(o is None for o in offs[k:]), (name, op, i, row)
            assert rest == sorted(rest), (name, op, i, row)
            if ring and n > 4:
                want = {-2, -1, 1, 2} if op == "laplacian" else {-1, 1}
                if op in ("gradient", "laplacian", "gradient_adjoint", "divergence_adjoint", "vector_gradient",
                          "divergence", "curl"):
                    assert want <= set(head), (name, op, i, row)


def test_group_tables_of_the_benchmark_grid_are_compact(product):
    """On O320 the merged entries per node (what the group kernels load) are
    4 against 6 per-node entries for the one-ring operators and 8.5 against
    18 for the two-ring Laplacian; no group has more than the 64 entries
    whose headers the kernels hold in registers."""
    atlas, _ = product
    fvm = atlas.build_fvm(320)
    for op, most in (("gradient", 0.67), ("divergence", 0.67), ("laplacian", 0.48)):
        st = fvm.stencil_table(op)
        gt = fvm.group_table(op)
        assert gt["hdr"].size < most * st["nbr"].size, op
        assert int(np.max(gt["head"][:, 2] - gt["head"][:, 1])) <= 64, op
