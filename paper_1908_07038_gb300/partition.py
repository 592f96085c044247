"""Band partitions of the grid's nodes with halo exchange, and level shards.

Atlas splits a mesh into partitions, one per MPI task, with overlap regions
refreshed by a halo exchange (paper Sec. 2.3).  Here a ``Partition`` wraps
``atlas_part_*``: part p of nparts owns the consecutive rows of one latitude
band, i.e. the node range [own0, own1), and its operators read the halo
range [halo0, halo1) = those rows plus 1 (2 for the fused Laplacian) rows on
each side.  A part's local field holds the halo range (row k = node
halo0 + k); ``exchange`` refreshes its halo rows from the two adjacent parts
with point-to-point messages of ``torch.distributed`` (rank = part index:
gloo for CPU tensors, NCCL for CUDA tensors), and the operator calls compute
the own nodes, bitwise equal to the whole-grid operators there.
``apply_overlapped`` hides the exchange behind computation (the asynchronous
communication the paper aims for, Sec. 2.2.3): the messages are started,
the interior nodes (whose stencils read no halo row) are computed, and the
rows next to the halo follow once the messages are done.

Levels are independent, so a field can instead be cut by levels with no
exchange at all: ``level_shards`` gives the level ranges (starting on 16-byte
boundaries), and the whole-grid calls take the column views.
"""
from __future__ import annotations

import ctypes

from . import capi
from .atlas import OPS, _dtype_code, _stream


class Partition:
    def __init__(self, fvm, nparts: int, part: int, halo_rings: int = 1):
        h = ctypes.c_void_p()
        capi.atlas_part_create(fvm.handle, int(nparts), int(part), int(halo_rings), ctypes.byref(h))
        self.handle, self.fvm = h, fvm
        self.nparts, self.part, self.halo_rings = int(nparts), int(part), int(halo_rings)
        v = [ctypes.c_int64() for _ in range(4)]
        capi.atlas_part_info(h, *(ctypes.byref(x) for x in v))
        self.own0, self.own1, self.halo0, self.halo1 = (x.value for x in v)
        self.neighbours = []
        for side in (0, 1):
            peer = ctypes.c_int()
            r = [ctypes.c_int64() for _ in range(4)]
            capi.atlas_part_neighbour(h, side, ctypes.byref(peer), *(ctypes.byref(x) for x in r))
            if peer.value >= 0:
                self.neighbours.append(dict(side=side, peer=peer.value, send=(r[0].value, r[1].value),
                                            recv=(r[2].value, r[3].value)))

    @property
    def local_rows(self):
        return self.halo1 - self.halo0

    @property
    def own_rows(self):
        return self.own1 - self.own0

    def local_view(self, field):
        """Rows [halo0, halo1) of a whole-grid field (for setting up tests)."""
        return field[self.halo0:self.halo1]

    def own_of_local(self, local):
        """The own rows inside a local field."""
        return local[self.own0 - self.halo0:self.own1 - self.halo0]

    def exchange_start(self, local, group=None):
        """Start sending this part's boundary rows to the adjacent parts and
        receiving their rows into the halo of ``local`` ([halo1 - halo0, ld],
        contiguous rows); returns the pending requests for ``exchange_wait``.
        Until then the halo rows must not be read, nor the sent rows written."""
        import torch.distributed as dist
        if local.shape[0] != self.local_rows or not local.is_contiguous():
            raise ValueError("local field must be contiguous with %d rows" % self.local_rows)
        reqs = []
        for n in self.neighbours:
            s0, s1 = (x - self.halo0 for x in n["send"])
            r0, r1 = (x - self.halo0 for x in n["recv"])
            reqs.append(dist.isend(local[s0:s1], n["peer"], group=group))
            reqs.append(dist.irecv(local[r0:r1], n["peer"], group=group))
        return reqs

    @staticmethod
    def exchange_wait(reqs):
        for r in reqs:
            r.wait()

    def exchange(self, local, group=None):
        """The exchange, blocking until its messages are done."""
        self.exchange_wait(self.exchange_start(local, group))

    @property
    def interior(self):
        """Own nodes [inner0, inner1) whose stencils read no halo row."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        capi.atlas_part_interior(self.handle, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def apply_overlapped(self, op, ins, outs, nlev=None, group=None):
        """Exchange the halos of ``ins`` while the interior nodes are
        computed, then compute the nodes next to the halo: the results of
        ``exchange`` followed by ``apply``, bitwise."""
        reqs = []
        for t in ins:
            reqs += self.exchange_start(t, group)
        i0, i1 = self.interior
        self.apply_nodes(op, ins, outs, i0, i1 - i0, nlev)
        self.exchange_wait(reqs)
        self.apply_nodes(op, ins, outs, self.own0, i0 - self.own0, nlev)
        self.apply_nodes(op, ins, outs, i1, self.own1 - i1, nlev)

    def apply(self, op, ins, outs, nlev=None):
        """Operator ``op`` on the own nodes: ins are local fields (halo rows
        filled), outs own-row fields; same dtype and leading dimension."""
        self.apply_nodes(op, ins, outs, self.own0, self.own_rows, nlev)

    def apply_nodes(self, op, ins, outs, node0, count, nlev=None):
        """``apply`` on the own nodes [node0, node0 + count) only (outs are
        still own-row fields; only those rows are written)."""
        ins, outs = list(ins), list(outs)
        t0 = ins[0]
        for t in ins:
            if t.shape[0] != self.local_rows:
                raise ValueError("inputs need %d rows (the halo range)" % self.local_rows)
        for t in outs:
            if t.shape[0] != self.own_rows:
                raise ValueError("outputs need %d rows (the own range)" % self.own_rows)
        for t in ins + outs:
            if not t.is_cuda or t.dim() != 2 or t.stride(1) != 1 or t.stride(0) != t0.stride(0) or t.dtype != t0.dtype:
                raise ValueError("fields must be CUDA tensors [rows, ld] of one dtype and leading dimension")
        p = [x.data_ptr() for x in ins] + [None] * (2 - len(ins))
        q = [x.data_ptr() for x in outs] + [None] * (2 - len(outs))
        capi.atlas_part_apply_nodes(self.handle, OPS.get(op, op), p[0], p[1], q[0], q[1], int(node0), int(count),
                                    t0.shape[1] if nlev is None else int(nlev), t0.stride(0), _dtype_code(t0),
                                    _stream())

    def integral(self, own, nlev=None, group=None, reduce=True):
        """FP64 volume-weighted sums over the own nodes of ``own`` (an
        own-row field, e.g. an output of ``apply``), added over all parts by
        ``torch.distributed.all_reduce`` when ``reduce``: the global
        conservation sums (0 for the divergence on the sphere).  The sum over
        parts adds one FP64 partial per part, so it can differ from the
        whole-grid integral by rounding."""
        if own.shape[0] != self.own_rows:
            raise ValueError("the field needs %d rows (the own range)" % self.own_rows)
        out = self.fvm.integral(own, nlev, node0=self.own0, count=self.own_rows)
        if reduce:
            import torch.distributed as dist
            dist.all_reduce(out, group=group)
        return out

    def close(self):
        if self.handle is not None and self.handle.value:
            capi.atlas_part_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def level_shards(nlev: int, nparts: int, align: int = 4):
    """Split levels [0, nlev) into nparts consecutive ranges of about equal
    size whose starts are multiples of ``align`` levels (16-byte boundaries
    for FP32), so that every shard keeps the vector loads."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    bounds = [0]
    for k in range(1, nparts):
        b = int(round(nlev * k / nparts / align)) * align
        bounds.append(min(max(b, bounds[-1]), nlev))
    bounds.append(nlev)
    return [(bounds[k], bounds[k + 1]) for k in range(nparts)]
