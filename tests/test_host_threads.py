"""The host side of the C ABI from several threads at once (ctypes releases the
interpreter lock for every foreign call, so the builds really overlap): grids,
meshes, duals and stencil tables built concurrently are bitwise equal to the
same objects built one after another, tables requested by several threads
from one fvm at the same time are built once and agree, and the last-error
text is per thread.  No GPU is used."""
import threading

import numpy as np
import pytest

R = 6371220.0
OPS = ("gradient", "divergence", "laplacian", "gradient_adjoint", "divergence_adjoint", "curl")


def _run(targets):
    """Run every callable on its own thread, started together; return the
    results in order and re-raise the first exception."""
    out = [None] * len(targets)
    errs = []
    start = threading.Barrier(len(targets))

    def body(k, fn):
        try:
            start.wait()
            out[k] = fn()
        except BaseException as e:  # noqa: BLE001 - handed to the main thread
            errs.append(e)

    ts = [threading.Thread(target=body, args=(k, fn)) for k, fn in enumerate(targets)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]
    return out


def _snapshot(fvm, ops=("gradient", "laplacian")):
    snap = {}
    for k, v in fvm.grid.arrays().items():
        snap["grid." + k] = np.array(v, copy=True)
    for k, v in fvm.mesh.arrays().items():
        snap["mesh." + k] = np.array(v, copy=True)
    for k, v in fvm.arrays().items():
        snap["dual." + k] = np.array(v, copy=True)
    for op in ops:
        for k, v in fvm.stencil_table(op).items():
            if isinstance(v, np.ndarray):
                snap[op + "." + k] = v.copy()
    return snap


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert a[k].dtype == b[k].dtype and np.array_equal(a[k], b[k]), k


def test_concurrent_global_builds_equal_serial_ones(product):
    atlas, _ = product
    Ns = (64, 96, 129, 160, 64, 129)
    serial = {N: _snapshot(atlas.build_fvm(N, R)) for N in set(Ns)}
    got = _run([lambda N=N: _snapshot(atlas.build_fvm(N, R)) for N in Ns])
    for N, snap in zip(Ns, got):
        _same(snap, serial[N])


def test_concurrent_regional_builds_equal_serial_ones(product):
    atlas, _ = product
    from synthetic.regional import DOMAINS
    names = ("rotated", "mercator", "lambert", "polar", "lambert", "rotated")

    def build(name):
        proj, kw = DOMAINS[name]
        return _snapshot(atlas.build_fvm_regional(proj, 29, 21, **kw), ops=OPS)

    serial = {n: build(n) for n in set(names)}
    got = _run([lambda n=n: build(n) for n in names])
    for n, snap in zip(names, got):
        _same(snap, serial[n])


def test_tables_of_one_fvm_requested_by_many_threads(product):
    atlas, _ = product
    ref = atlas.build_fvm(20, R)
    want = {op: {k: v.copy() for k, v in ref.stencil_table(op).items() if isinstance(v, np.ndarray)} for op in OPS}
    fvm = atlas.build_fvm(20, R)
    ops = OPS * 3
    got = _run([lambda op=op: fvm.stencil_table(op) for op in ops])
    for op, tab in zip(ops, got):
        for k, v in want[op].items():
            assert np.array_equal(tab[k], v), (op, k)


def test_last_error_is_per_thread(product):
    """Each thread's failing call reports its own argument, although the
    other threads fail (or succeed) at the same time."""
    atlas, capi = product
    bad = (-7, 0, 9001, 12345, -1, 8001)

    def fail(N):
        with pytest.raises(capi.AtlasError) as ei:
            atlas.build_fvm(N, R)
        return str(ei.value)

    def succeed():
        return atlas.build_fvm(12, R).nnodes

    got = _run([lambda N=N: fail(N) for N in bad] + [succeed, succeed])
    for N, msg in zip(bad, got):
        assert ("N=%d " % N) in msg, msg
    assert got[-1] == got[-2] == atlas.build_fvm(12, R).nnodes
