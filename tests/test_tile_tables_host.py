"""Host checks of the node-group kernels' tile tables (no GPU).

A tile stages the node rows its groups read in shared memory and carries a
table per group in one of two forms.  The kernels read it as follows.
  * Per-node form: for entry e, one slot and one weight pair per node of
    the group.
  * Union form (groups of four whose union of stencil rows matches the
    operator's pattern in patterns.h): one slot per distinct neighbour,
    applied to the nodes of the pattern's mask for that entry, in node
    order, each consuming its next weights.
These tests decode both forms the way the kernels do and check that every
node meets exactly its own stencil row, in its order, with its FP32
weights.  The union form is also checked against the compiled pattern
(masks, and the entries that are the group's own nodes, which the kernels
take from registers), and its coverage on octahedral grids is checked.
"""
import os
import re

import numpy as np
import pytest

OPS = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint", "curl", "vector_gradient")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _patterns():
    """The compiled union patterns: {name: (U, RUN0, NRUN, masks)}."""
    src = open(os.path.join(ROOT, "paper_1908_07038_gb300", "csrc", "patterns.h")).read()
    out = {}
    for name, body in re.findall(r"struct (Ring\d) \{(.*?)\};", src, re.S):
        u = int(re.search(r"U = (\d+)", body).group(1))
        run0 = int(re.search(r"RUN0 = (-?\d+)", body).group(1))
        nrun = int(re.search(r"NRUN = (\d+)", body).group(1))
        masks = [int(c, 16) for c in re.search(r'hexval\("([0-9a-f]+)"', body).group(1)]
        assert len(masks) == u
        out[name] = (u, run0, nrun, masks)
    return out


@pytest.fixture(scope="module")
def fvms(product):
    atlas, _ = product
    from synthetic.regional import DOMAINS
    proj, kw = DOMAINS["lambert"]
    return {"O2": atlas.build_fvm(2), "O24": atlas.build_fvm(24), "O64": atlas.build_fvm(64),
            "F6": atlas.build_fvm(6, regular=True),
            "lambert13x9": atlas.build_fvm_regional(proj, 13, 9, **kw)}


def _f32(words):
    return np.asarray(words, np.uint32).view(np.float32)


def _decode(fvm, op, groups_per_tile, unions, rows_per_tile=1):
    """Per node: the (neighbour, weights) terms the kernels apply, in order;
    the number of union groups and of tiles.  Also checks the units: runs
    of whole grid rows whose consecutive tiles hold exactly their nodes."""
    st = fvm.stencil_table(op)
    tt = fvm.tile_table(op, groups_per_tile, unions, rows_per_tile)
    head, blob, uf, ut = tt["head"], tt["blob"], tt["unit_first"], tt["unit_tile"]
    nw = 1 if op == "laplacian" else 2
    ptr, nbr = st["ptr"], st["nbr"]
    pats = _patterns()
    pat = pats["Ring2"] if op == "laplacian" else pats["Ring1"]
    V = fvm.nnodes
    terms = [None] * V
    nuni = 0
    covered = 0
    off = np.concatenate([[0], np.cumsum(fvm.grid.arrays()["pl"])])
    assert uf[0] == 0 and uf[-1] == V and np.all(np.diff(uf) > 0) and np.all(np.isin(uf, off))
    assert ut[0] == 0 and ut[-1] == head.shape[0] and np.all(np.diff(ut) > 0)
    unit_of_tile = np.repeat(np.arange(len(ut) - 1), np.diff(ut))
    rows_of_unit = np.diff(np.searchsorted(off, uf))
    assert np.all(rows_of_unit <= rows_per_tile)
    for t in range(head.shape[0]):
        h = head[t]
        first, ngt, nr, nslots, boff, bbytes = (int(x) for x in h[:6])
        ids = np.full(nslots, -1, np.int64)
        for r in range(nr):
            rf, rc, rs = (int(x) for x in h[8 + 4 * r: 11 + 4 * r])
            ids[rs:rs + rc] = np.arange(rf, rf + rc)
        assert np.all(ids >= 0) and np.all(np.diff(ids) > 0)  # slot s: the s-th smallest id
        b = blob[4 * boff: 4 * boff + bbytes // 4]
        assert int(b[0]) == ngt and int(b[2]) == first and 1 <= ngt <= groups_per_tile
        u_t = unit_of_tile[t]
        for k in range(ngt):
            slot0, off, node0, flags = (int(x) for x in b[4 + 4 * k: 8 + 4 * k])
            cnt, regular, uni, D = flags & 0xFFFF, (flags >> 16) & 1, (flags >> 17) & 1, (flags >> 20) & 0xFF
            assert flags >> 28 == 0 and (flags >> 18) & 3 == 0
            assert ids[slot0] == node0 and uf[u_t] <= node0 and node0 + cnt <= uf[u_t + 1]
            assert terms[node0] is None  # every node in one group of one tile
            nodes = [node0 + u for u in range(cnt)]
            rows = [list(nbr[ptr[i]:ptr[i + 1]]) for i in nodes]
            got = [[] for _ in nodes]
            if uni:
                U, run0, nrun, masks = pat
                assert unions and cnt == 4 and regular and D == U
                sl = b[off: off + U]
                wv = _f32(b[off + ((U + 3) & ~3):])
                p = 0
                for e in range(U):
                    j = int(ids[sl[e]]) if e >= nrun or not 0 <= run0 + e < 4 else node0 + run0 + e
                    if e < nrun and 0 <= run0 + e < 4:
                        assert int(ids[sl[e]]) == j  # the group's own node: taken from registers
                    m = sum(1 << u for u in range(4) if j in rows[u])
                    assert m == masks[e], (t, k, e)
                    for u in range(4):
                        if m >> u & 1:
                            got[u].append((j, tuple(wv[p:p + nw])))
                            p += nw
                assert p == sum(bin(x).count("1") for x in masks) * nw
                nuni += 1
            else:
                sl = b[off: off + 4 * D].reshape(D, 4)
                wv = _f32(b[off + 4 * D: off + 4 * D * (1 + 2 * nw)]).reshape(D, 4, nw, 2)
                assert np.all(wv[..., 0] == wv[..., 1])  # each weight twice
                for u in range(4):
                    i = node0 + min(u, cnt - 1)
                    deg = ptr[i + 1] - ptr[i] if u < cnt else 0
                    for e in range(D):
                        if e < deg:
                            got[u].append((int(ids[sl[e, u]]), tuple(wv[e, u, :, 0])))
                        else:
                            assert ids[sl[e, u]] == i and np.all(wv[e, u] == 0)
                if regular:
                    R, off_r = (4, (-2, -1, 1, 2)) if op == "laplacian" else (2, (-1, 1))
                    assert cnt == 4 and D >= R
                    for u in range(4):
                        for r in range(R):
                            if 0 <= u + off_r[r] < 4:
                                assert ids[sl[r, u]] == node0 + u + off_r[r]
            for u, i in enumerate(nodes):
                terms[i] = got[u]
            covered += cnt
    assert covered == V
    return terms, nuni, head.shape[0]


@pytest.mark.parametrize("name", ["O2", "O24", "F6", "lambert13x9"])
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("unions,rows,groups", [(True, 1, 7), (False, 1, 7), (True, 2, 8), (False, 2, 4),
                                                (True, 3, 6), (True, 2, 10), (True, 2, 12), (True, 1, 15)])
def test_tile_tables_give_every_node_its_row(fvms, name, op, unions, rows, groups):
    fvm = fvms[name]
    st = fvm.stencil_table(op)
    nw = 1 if op == "laplacian" else 2
    terms, nuni, _ = _decode(fvm, op, groups, unions, rows)
    ptr, nbr, w = st["ptr"], st["nbr"], st["w"]
    for i in range(fvm.nnodes):
        want = [(int(nbr[q]), tuple(np.float32(w[q, c]) for c in range(nw))) for q in range(ptr[i], ptr[i + 1])]
        assert terms[i] == want, i
    if not unions:
        assert nuni == 0


@pytest.mark.parametrize("op", ["gradient", "laplacian", "divergence"])
def test_union_groups_cover_octahedral_interiors(fvms, op):
    # the patterns are those of an octant's interior: most groups of an
    # octahedral grid take the union form, more of them on finer grids
    frac = {}
    for name in ("O24", "O64"):
        _, n, _ = _decode(fvms[name], op, 11, True)
        frac[name] = n / sum(-(-p // 4) for p in fvms[name].grid.arrays()["pl"])
    assert frac["O64"] > frac["O24"] and frac["O64"] > (0.8 if op == "laplacian" else 0.85), frac


def test_multi_row_tiles_stage_fewer_rows(fvms):
    # a tile spanning two grid rows stages the rows above and below once for
    # both: fewer staged rows per node than tiles of one row
    def per_node(op, groups, rows):
        tt = fvms["O64"].tile_table(op, groups, True, rows)
        return tt["head"][:, 3].sum() / fvms["O64"].nnodes
    assert per_node("laplacian", 8, 2) < 0.75 * per_node("laplacian", 4, 1)
    assert per_node("divergence", 8, 2) < 0.8 * per_node("divergence", 7, 1)


def test_tile_table_arguments(fvms):
    from paper_1908_07038_gb300.capi import AtlasError
    with pytest.raises(AtlasError):
        fvms["O2"].tile_table("gradient", 16)
    with pytest.raises(AtlasError):
        fvms["O2"].tile_table("gradient", 0)
    with pytest.raises(AtlasError):
        fvms["O2"].tile_table("gradient", 4, True, 4)
