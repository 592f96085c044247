"""Host side of the batched launch, on CPU: the seeded job mix, and the
argument checks of ``atlas_batch_create`` that come before the device (a
batch on a machine without a GPU is refused, never run on the CPU)."""
import pytest


EINVAL, ECUDA, EDTYPE = -1, -3, -5
SMALL = (8, 12, 16, 20)  # the job mix over small grids (the benchmark's are O80-O640)


@pytest.fixture
def fvms(pfvm, product, monkeypatch):
    from paper_1908_07038_gb300 import batch
    monkeypatch.setattr(batch, "GRIDS", SMALL)
    return {N: pfvm(N) for N in SMALL}


def test_job_mix_is_seeded_and_padded(fvms, product):
    torch = pytest.importorskip("torch")
    from paper_1908_07038_gb300 import batch
    a = batch.make_jobs(fvms, 12, seed=3, device="cpu")
    b = batch.make_jobs(fvms, 12, seed=3, device="cpu")
    c = batch.make_jobs(fvms, 12, seed=4, device="cpu")
    assert [j["op"] for j in a] == ["gradient", "divergence"] * 6
    for ja, jb in zip(a, b):
        assert (ja["N"], ja["nlev"]) == (jb["N"], jb["nlev"])
        for x, y in zip(ja["ins"], jb["ins"]):
            assert torch.equal(x, y)
    assert [(j["N"], j["nlev"]) for j in a] != [(j["N"], j["nlev"]) for j in c]
    for j in a:
        assert j["N"] in SMALL and j["nlev"] in batch.LEVELS
        t = j["ins"][0]
        assert t.dtype == torch.float32 and t.shape[0] == j["fvm"].nnodes
        ld = t.stride(0)
        assert ld % 4 == 0 and j["nlev"] <= ld < j["nlev"] + 4
        assert torch.count_nonzero(t[:, j["nlev"]:]) == 0  # padding levels are zero
        for o in j["outs"]:
            assert o.shape == t.shape


def test_batch_without_a_gpu_is_refused(fvms, product):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    _, capi = product
    from paper_1908_07038_gb300 import batch
    jobs = batch.make_jobs(fvms, 4, seed=3, device="cpu")
    with pytest.raises(capi.AtlasError) as ei:
        batch.Batch(jobs)
    assert ei.value.code == ECUDA


def test_batch_argument_checks(fvms, product):
    torch = pytest.importorskip("torch")
    _, capi = product
    from paper_1908_07038_gb300 import batch
    jobs = batch.make_jobs(fvms, 4, seed=3, device="cpu")
    mixed = list(jobs)
    mixed[1] = dict(mixed[1], ins=tuple(x.double() for x in mixed[1]["ins"]))
    with pytest.raises(ValueError):
        batch.Batch(mixed)
    for tune, code in ((dict(vec=3), EINVAL), (dict(threads=48), EINVAL),
                       (dict(threads=100), EINVAL), (dict(plain_waves=-2), EINVAL)):
        with pytest.raises(capi.AtlasError) as ei:
            batch.Batch(jobs, tune=tune)
        assert ei.value.code == code, tune
    bf = [dict(j, ins=tuple(x.to(torch.bfloat16) for x in j["ins"])) for j in jobs]
    with pytest.raises(capi.AtlasError) as ei:
        batch.Batch(bf)
    assert ei.value.code == EDTYPE
    with pytest.raises(ValueError):
        batch.Batch([])
    import ctypes
    h = ctypes.c_void_p()
    with pytest.raises(capi.AtlasError) as ei:  # the C call refuses an empty table too
        capi.atlas_batch_create(None, 0, 0, None, ctypes.byref(h))
    assert ei.value.code == EINVAL
