"""The five nabla operators applied to fields that live in pinned host memory.

``HostStep`` owns device copies of the inputs (f, u, v) and of the seven
outputs and runs one step as

    host f, u, v --H2D--> device --kernels--> device --D2H--> host outputs

on three CUDA streams (copy-in, compute, copy-out) ordered by events.  Each
operator starts as soon as its own inputs are on the device and each result
is copied out as soon as its operator has finished, so the link carries the
inputs of one operator and the outputs of another while the kernels run.
Consecutive steps overlap the same way: the copy-in of the next step's field
waits only for the kernels that read the previous one, and a kernel waits
only for the copy-out of the buffer it overwrites.  With the kernels about
ten times faster than the host link, a step costs about the link time of its
bytes.  Every copy is one ``atlas_field_sync`` (one ``cudaMemcpyAsync``);
every operator is its ``atlas_nabla_*`` entry point.
"""
from __future__ import annotations

from . import atlas

# operator -> (inputs, outputs) by name
IO = {
    "gradient": (("f",), ("gx", "gy")),
    "laplacian": (("f",), ("lap",)),
    "divergence_adjoint": (("f",), ("du", "dv")),
    "divergence": (("u", "v"), ("div",)),
    "gradient_adjoint": (("u", "v"), ("ga",)),
}
INPUTS = ("f", "u", "v")
OUTPUTS = ("gx", "gy", "lap", "du", "dv", "div", "ga")


class HostStep:
    """Pipelined host-to-host application of the operators in ``ops``.

    fvm: the Fvm; nnodes x ld fields of torch dtype ``dtype`` with nlev levels.
    ops: operators to apply, in launch order (default: the f operators first,
    since f is copied first).
    """

    def __init__(self, fvm, nlev, ld, dtype, ops=tuple(IO)):
        torch = atlas._torch()
        self.torch = torch
        self.fvm, self.nlev, self.ld, self.ops = fvm, int(nlev), int(ld), tuple(ops)
        for op in self.ops:
            if op not in IO:
                raise ValueError("unknown operator %r" % op)
        need_in = [n for n in INPUTS if any(n in IO[op][0] for op in self.ops)]
        need_out = [n for op in self.ops for n in IO[op][1]]
        shape = (fvm.nnodes, self.ld)
        self.dev = {n: torch.empty(shape, dtype=dtype, device="cuda") for n in need_in + need_out}
        self.inputs, self.outputs = tuple(need_in), tuple(need_out)
        self.nbytes = fvm.nnodes * self.ld * self.dev[need_in[0]].element_size()
        self.s_in, self.s_comp, self.s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        E = torch.cuda.Event
        self.ev_in = {n: E() for n in need_in}          # input n is on the device
        self.ev_read = {n: E() for n in need_in}        # last kernel reading input n has finished
        self.ev_done = {op: E() for op in self.ops}     # operator finished
        self.ev_out = {n: E() for n in need_out}        # output n is back on the host
        self._first = True

    @property
    def h2d_bytes(self):
        return len(self.inputs) * self.nbytes

    @property
    def d2h_bytes(self):
        return len(self.outputs) * self.nbytes

    def _check_host(self, t):
        if t.device.type != "cpu" or t.shape != (self.fvm.nnodes, self.ld) or t.dtype != self.dev[self.inputs[0]].dtype:
            raise ValueError("host buffers must be CPU tensors of shape %r and the step's dtype" %
                             ((self.fvm.nnodes, self.ld),))
        if not t.is_contiguous():
            raise ValueError("host buffers must be contiguous")

    def enqueue(self, host_in, host_out):
        """Enqueue one step; returns at once.  host_in / host_out: dicts of
        pinned CPU tensors by name (INPUTS / OUTPUTS).  The host outputs are
        complete once ``synchronize`` (or the copy-out stream) says so."""
        torch = self.torch
        for n in self.inputs:
            self._check_host(host_in[n])
        for n in self.outputs:
            self._check_host(host_out[n])
        first = self._first
        self._first = False
        # copy-in: input n may be overwritten once the kernels reading it are done
        for n in self.inputs:
            if not first:
                self.s_in.wait_event(self.ev_read[n])
            atlas.field_sync(self.dev[n].data_ptr(), host_in[n].data_ptr(), self.nbytes, 0, self.s_in.cuda_stream)
            self.ev_in[n].record(self.s_in)
        fvm, nlev, d = self.fvm, self.nlev, self.dev
        last_reader = {}
        for op in self.ops:
            ins, outs = IO[op]
            for n in ins:
                self.s_comp.wait_event(self.ev_in[n])
            if not first:
                for n in outs:
                    self.s_comp.wait_event(self.ev_out[n])
            with torch.cuda.stream(self.s_comp):
                if op == "gradient":
                    fvm.gradient(d["f"], nlev, out=(d["gx"], d["gy"]))
                elif op == "laplacian":
                    fvm.laplacian(d["f"], nlev, out=d["lap"])
                elif op == "divergence_adjoint":
                    fvm.divergence_adjoint(d["f"], nlev, out=(d["du"], d["dv"]))
                elif op == "divergence":
                    fvm.divergence(d["u"], d["v"], nlev, out=d["div"])
                else:
                    fvm.gradient_adjoint(d["u"], d["v"], nlev, out=d["ga"])
            self.ev_done[op].record(self.s_comp)
            for n in ins:
                last_reader[n] = op
            # copy-out of this operator's results
            self.s_out.wait_event(self.ev_done[op])
            for n in outs:
                atlas.field_sync(host_out[n].data_ptr(), d[n].data_ptr(), self.nbytes, 1, self.s_out.cuda_stream)
                self.ev_out[n].record(self.s_out)
        for n in self.inputs:
            self.ev_read[n] = self.ev_done[last_reader[n]]

    def begin(self, stream=None):
        """Order everything enqueued from now on after the work already on
        ``stream`` (default: torch's current stream)."""
        s = stream if stream is not None else self.torch.cuda.current_stream()
        for t in (self.s_in, self.s_comp, self.s_out):
            t.wait_stream(s)

    def join(self, stream=None):
        """Make ``stream`` (default: torch's current stream) wait for every
        copy and kernel enqueued so far."""
        s = stream if stream is not None else self.torch.cuda.current_stream()
        s.wait_stream(self.s_in)
        s.wait_stream(self.s_comp)
        s.wait_stream(self.s_out)

    def synchronize(self):
        self.s_in.synchronize()
        self.s_comp.synchronize()
        self.s_out.synchronize()

    def run(self, host_in, host_out):
        """One step, returned when the host outputs are complete."""
        self.enqueue(host_in, host_out)
        self.synchronize()
